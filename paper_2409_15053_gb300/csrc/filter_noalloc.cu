// flz_filter_apply_noalloc: the FP64 filter W = p_m((A - cI)/e) V for callers
// that cannot allocate device memory.
//
// Who needs it: code whose device memory is owned by someone else's pool (a
// framework's caching allocator that has reserved the GPU, or an embedding
// application with a fixed memory budget) and latency-sensitive callers that
// cannot afford cudaMalloc/cudaFree, which synchronize the whole device. Such
// callers hold the CSR arrays and the V / W blocks already; the only extra
// memory the filter needs is two n x r recurrence buffers, and here those come
// from a fixed, file-scope device array instead of an allocation.
//
// The array is kNoAllocElems x 2 doubles (16 MiB) and lives in every GPU that
// loads this library until the process exits. Host code cannot use its name as
// an address (on the host it names a stand-in object), so the entry point asks
// the runtime for the device address with cudaGetSymbolAddress once per device,
// on its first call on that device, and passes that address to the kernels.
// The first call on each device should therefore be made before any stream
// capture begins. All calls share the array: calls that overlap in time on the
// GPU (different streams, different threads) race on it and must be ordered by
// the caller. Nothing in the array needs to start at zero: every recurrence
// buffer element is written before it is read within one call.
#include <mutex>

#include "flz_internal.h"

namespace {

constexpr long long kNoAllocElems = 1LL << 20;  // per recurrence buffer: n * r <= 1,048,576
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocElems];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set up once per device).
double* scratch_address() {
  int dev = 0;
  FLZ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) flz::fail(FLZ_ERR_INVALID_ARG, "device index %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess || p == nullptr)
      flz::fail(FLZ_ERR_CUDA, "cudaGetSymbolAddress of the filter scratch failed: %s", cudaGetErrorString(err));
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
}

// One fused Chebyshev step in FP64 (same arithmetic as the library's filter):
//   Y_next = alpha (A Y_cur) + beta Y_cur - (first ? 0 : Y_prev)
//   acc    = (first ? b_cur Y_cur : acc) + b_next Y_next
// r lanes per row, 32/r rows per warp. ynext may alias yprev, acc_out acc_in.
template <bool FIRST>
__global__ void __launch_bounds__(kThreads) noalloc_step_kernel(int n, int r, int rows_per_warp,
                                                                const int* __restrict__ rowptr,
                                                                const int* __restrict__ col,
                                                                const double* __restrict__ val,
                                                                const double* __restrict__ ycur,
                                                                const double* yprev, double* ynext,
                                                                const double* acc_in, double* acc_out, double alpha,
                                                                double beta, double b_cur, double b_next) {
  const int lane = threadIdx.x & 31;
  const int sub = lane / r;
  const int c = lane - sub * r;
  const long long row = (((long long)blockIdx.x * kThreads + threadIdx.x) >> 5) * rows_per_warp + sub;
  if (sub >= rows_per_warp || row >= n) return;
  double s = 0.0;
  for (int j = __ldg(rowptr + row), je = __ldg(rowptr + row + 1); j < je; ++j)
    s = fma(__ldg(val + j), ycur[(size_t)__ldg(col + j) * r + c], s);
  const size_t idx = (size_t)row * r + c;
  const double yc = ycur[idx];
  double yn = fma(alpha, s, beta * yc);
  if (!FIRST) yn -= yprev[idx];
  ynext[idx] = yn;
  const double acc = FIRST ? b_cur * yc : acc_in[idx];
  acc_out[idx] = fma(b_next, yn, acc);
}

__global__ void noalloc_scale_kernel(const double* __restrict__ in, double* __restrict__ out, double s,
                                     long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = s * in[i];
}

}  // namespace

extern "C" flz_status flz_filter_apply_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                               const double* val, double c, double e, const double* coeffs,
                                               int32_t degree, int32_t r, const double* V, double* W,
                                               void* stream) {
  flz::clear_last_error();
  try {
    if (!rowptr || !coeffs || !V || !W || (nnz > 0 && (!col || !val)))
      flz::fail(FLZ_ERR_INVALID_ARG, "null argument");
    if (n < 1 || nnz < 0 || n > 2147483647LL || nnz > 2147483647LL) flz::fail(FLZ_ERR_INVALID_ARG, "n/nnz out of range");
    if (degree < 0 || r < 1 || r > 16 || !(e > 0.0)) flz::fail(FLZ_ERR_INVALID_ARG, "need degree >= 0, 1 <= r <= 16, e > 0");
    const long long nr = n * (long long)r;
    if (nr > kNoAllocElems)
      flz::fail(FLZ_ERR_CAPACITY, "n*r = %lld exceeds the fixed scratch of %lld elements per buffer", nr, kNoAllocElems);
    const char* v = reinterpret_cast<const char*>(V);
    const char* w = reinterpret_cast<const char*>(W);
    const size_t bytes = sizeof(double) * (size_t)nr;
    if (v < w + bytes && w < v + bytes) flz::fail(FLZ_ERR_INVALID_ARG, "V and W overlap");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (degree == 0) {
      const unsigned grid = (unsigned)std::min<long long>((nr + 255) / 256, 152 * 16);
      noalloc_scale_kernel<<<grid, 256, 0, st>>>(V, W, coeffs[0], nr);
      FLZ_LAUNCH_CHECK();
      return FLZ_OK;
    }
    double* scratch = scratch_address();
    double* ya = scratch;
    double* yb = scratch + kNoAllocElems;
    const int rpw = 32 / r;
    const long long warps = (n + rpw - 1) / rpw;
    const unsigned grid = (unsigned)((warps * 32 + kThreads - 1) / kThreads);
    const int ni = (int)n;
    noalloc_step_kernel<true><<<grid, kThreads, 0, st>>>(ni, r, rpw, rowptr, col, val, V, nullptr, ya, nullptr, W,
                                                         1.0 / e, -c / e, coeffs[0], coeffs[1]);
    FLZ_LAUNCH_CHECK();
    const double* prev = V;
    const double* cur = ya;
    for (int k = 1; k < degree; ++k) {
      double* next = (k == 1) ? yb : const_cast<double*>(prev);
      noalloc_step_kernel<false><<<grid, kThreads, 0, st>>>(ni, r, rpw, rowptr, col, val, cur, prev, next, W, W,
                                                            2.0 / e, -2.0 * c / e, 0.0, coeffs[k + 1]);
      FLZ_LAUNCH_CHECK();
      prev = cur;
      cur = next;
    }
    return FLZ_OK;
  } catch (const flz::Failure& f) {
    return f.status;
  } catch (...) {
    flz::set_last_error("unexpected internal error");
    return FLZ_ERR_CUDA;
  }
}
