// Internal declarations shared by the translation units of libflz.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "flz.h"
#include "device_common.cuh"

namespace flz {

// Internal failures are C++ exceptions carrying a status; every extern "C"
// entry point catches them, so nothing crosses the ABI.
struct Failure {
  flz_status status;
};

[[noreturn]] void fail(flz_status st, const char* fmt, ...);
// Limit of every bounded device-side wait of kernels launched from now on
// (flz_set_wait_limit; 2 s by default).
uint64_t wait_limit_ns();
extern std::atomic<uint64_t> g_wait_ns;
void set_last_error(const char* msg);
void clear_last_error();

#define FLZ_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      ::flz::fail(e_ == cudaErrorMemoryAllocation ? FLZ_ERR_OUT_OF_MEMORY : FLZ_ERR_CUDA,    \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

// Every kernel launch site is followed by FLZ_LAUNCH_CHECK(), which also
// counts the launch (reported per solve in flz_stats.kernel_launches).
extern thread_local int64_t g_kernel_launches;
#define FLZ_LAUNCH_CHECK()         \
  do {                             \
    ++::flz::g_kernel_launches;    \
    FLZ_CUDA(cudaGetLastError());  \
  } while (0)

// Launches kernel K with programmatic stream serialization: it may begin (and
// run its prologue up to grid_dependency_wait()) while the previous kernel on
// the stream is still finishing.
template <class... P, class... Args>
inline void launch_dependent(void (*K)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FLZ_CUDA(cudaLaunchKernelEx(&cfg, K, static_cast<P>(args)...));
}

// Entry-point bodies: clear the thread's last error, run, map failures to a status.
#define FLZ_API_BEGIN         \
  ::flz::clear_last_error();  \
  try {
#define FLZ_API_END                                     \
  }                                                     \
  catch (const ::flz::Failure& f) {                     \
    return f.status;                                    \
  }                                                     \
  catch (const std::bad_alloc&) {                       \
    ::flz::set_last_error("host allocation failed");    \
    return FLZ_ERR_OUT_OF_MEMORY;                       \
  }                                                     \
  catch (...) {                                         \
    ::flz::set_last_error("unexpected internal error"); \
    return FLZ_ERR_CUDA;                                \
  }                                                     \
  return FLZ_OK;

// Owning device buffer.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t count = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    count = 0;
  }
  // Ensures capacity for n elements; contents are not preserved on growth.
  void reserve(size_t n) {
    if (n <= count && p) return;
    release();
    if (n == 0) return;
    FLZ_CUDA(cudaMalloc(reinterpret_cast<void**>(&p), n * sizeof(T)));
    count = n;
  }
};

// ---- tc_ortho.cu ----------------------------------------------------------------
// The Krylov basis as eight BF16-exact base-256 digits per value (64-bit fixed
// point, 2^-62 units) for full reorthogonalization on the tensor cores, with
// the scratch of its projection and update kernels. Columns are appended
// block by block; appending rounds the FP64 block to the same 2^-62 grid so
// the FP64 and digit copies hold the same numbers.
struct TcBasis {
  DevBuf<uint8_t> q;        // digit strips, zero outside the written columns and rows
  DevBuf<unsigned long long> acc;  // projection sums per group (128 x N each), zero between projections
  DevBuf<uint8_t> wd;       // digits of the block being projected (n_pad x N x 2 bytes)
  DevBuf<uint16_t> hs;      // digits of the coefficient matrix of an update
  DevBuf<int> hexp;         // its column scale exponents
  DevBuf<uint32_t> wmax;    // column maxima of W (two sets of 16)
  DevBuf<int> status;       // first failed wait of any launch (0 = none)
  int* status_host = nullptr;  // pinned copy, refreshed at the end of every cgs2
  int64_t n = 0, n_pad = 0, n_oct = 0;
  int groups_cap = 0;
  TcBasis() = default;
  TcBasis(const TcBasis&) = delete;
  TcBasis& operator=(const TcBasis&) = delete;
  ~TcBasis() { release(); }
  static bool supported(int r);                       // block widths the kernels take (1..16)
  static size_t bytes_for(int64_t n, int64_t kcap);   // digit storage for kcap columns
  void release();
  void reserve(int64_t n, int64_t kcap);
  // room for kcap columns, keeping the digits written so far (at least doubles the capacity)
  void grow(int64_t kcap, cudaStream_t st);
  // an empty digit basis of n rows and kcap columns in the allocation already
  // held when it is large enough (zeroed on st), else a new one
  void reshape(int64_t n, int64_t kcap, cudaStream_t st);
  // rounds X (n x r, row-major) to the 2^-62 grid in place; its digits become columns col0..col0+r-1
  void append(double* X, int r, int col0, cudaStream_t st);
  // out[j] = largest |W[i, j]| (as the upper word of the FP64 bits), j < r
  void column_max(const double* W, int r, int ldw, uint32_t* out, cudaStream_t st);
  // C[kb, j] = sum_i Q[i, kb] W[i, j], kb < K (row stride ldc), from W's digits at the scales in wmax
  void project(int K, const double* W, int r, int ldw, const uint32_t* wmax, double* C, int ldc, cudaStream_t st);
  // W -= Q[:, :K] C; records the new column maxima of W in wmax_out if not null
  void subtract(int K, const double* C, int ldc, double* W, int r, int ldw, uint32_t* wmax_out, cudaStream_t st);
  // X[:, :s] = Q[:, :K] C (C K x s with row stride ldc, X row stride ldx), eight columns per pass
  void multiply(int K, const double* C, int ldc, int s, double* X, int ldx, cudaStream_t st);
  // classical Gram-Schmidt twice of W (n x r) against columns 0..K-1; C, C2 the two projections
  void cgs2(int K, double* W, int r, double* C, double* C2, cudaStream_t st);
  // raises FLZ_ERR_TIMEOUT if a kernel recorded an expired wait (after a stream sync)
  void check_status();
};
// One tcgen05 MMA (M = 128, N = np, K = 16, BF16 in, FP32 out) of shared-memory
// images with explicit descriptor strides; out is 128 x np row-major. Returns
// the kernel's wait status (0 = completed).
int tc_probe(const uint16_t* a_img, size_t a_bytes, const uint16_t* b_img, size_t b_bytes, int np, int a_mn_major,
             uint32_t a_lbo, uint32_t a_sbo, uint32_t b_lbo, uint32_t b_sbo, float* out_host);

}  // namespace flz

namespace flz {
// State of the 64-bit fixed-point filter on a matrix handle: 2 Ahat as
// offset-binary integers (units 2^-61) in CSR order (slot 0) and in the
// SELL-32 layout (slot 1) for the (c, e) they were built for, the largest
// absolute row sum of 2 Ahat, the recurrence scratch and a few device words
// (column exponents, overflow flag).
struct FxValues {
  DevBuf<uint64_t> csr, sell, ws, scratch;
  DevBuf<double> part;
  double c[2] = {0.0, 0.0}, e[2] = {0.0, 0.0}, rowsum[2] = {0.0, 0.0};
  bool ok[2] = {false, false};
  unsigned* flag_host = nullptr;
  FxValues() = default;
  FxValues(const FxValues&) = delete;
  FxValues& operator=(const FxValues&) = delete;
  ~FxValues() {
    if (flag_host) cudaFreeHost(flag_host);
  }
};

// The fixed-point filter of a batch (the block-diagonal concatenation of its
// problems): SELL-32 layout of the concatenation, its values 2 Ahat_i in each
// problem's own map, per-problem coefficient tables and the recurrence
// vectors.
struct FxBatch {
  bool layout_built = false, layout_ok = false;
  int64_t n = 0, nsl = 0, emax = 0;
  DevBuf<int32_t> sell_off, sell_col;
  DevBuf<uint64_t> sval, y0, ya, yb, bfix;
  DevBuf<int> sexp, zexp, cta_p0;
  DevBuf<unsigned> flag, gbar;
  unsigned* flag_host = nullptr;
  int vec_bits = 61, mmax = 0, count = 0;
  int rows = 256;  // rows per CTA of the degree-step kernel (128 or 256; the batch autotuner's choice)
  double rowsum = 0.0;
  FxBatch() = default;
  FxBatch(const FxBatch&) = delete;
  FxBatch& operator=(const FxBatch&) = delete;
  ~FxBatch() {
    if (flag_host) cudaFreeHost(flag_host);
  }
};
}  // namespace flz

// Matrix handle: a device copy of a symmetric CSR matrix (Section 3.2.1).
struct flz_matrix {
  int64_t n = 0, nnz = 0;              // nnz counts the stored entries (explicit zero diagonals included)
  int64_t nnz_user = 0;                // entries the caller passed
  int device = 0;
  flz::DevBuf<int32_t> rowptr, col;
  flz::DevBuf<double> val;
  flz::DevBuf<int32_t> diag_pos;       // position of a_ii in col/val for every row
  // 2 Ahat = (2/e)(A - cI) in each filter storage precision (FP64, FP32, BF16),
  // rebuilt when (c, e) change: the filter kernels read only these values.
  flz::DevBuf<double> sval64;
  flz::DevBuf<float> sval32;
  flz::DevBuf<__nv_bfloat16> sval16;
  flz::DevBuf<flz::dev::dfloat> svaldf;  // double-FP32 (hi, lo) values
  double sc_c[4] = {0.0, 0.0, 0.0, 0.0}, sc_e[4] = {0.0, 0.0, 0.0, 0.0};
  bool sc_ok[4] = {false, false, false, false};
  double glo = 0.0, ghi = 0.0;         // Gershgorin interval
  int32_t max_row_nnz = 0;
  int32_t max_cta_nnz = 0;             // most stored entries in any 256 consecutive rows
  flz::DevBuf<int32_t> long_rows;      // rows with more than kLongRow entries (filter's CTA-per-row tier)
  int32_t n_long = 0;
  // SELL-32 copy of the structure for the filter (sliced ELLPACK: slice s =
  // rows 32s..32s+31, entry j of lane l at sell_off[s] + 32 j + l; padding
  // has column = own row and value 0; a row longer than kLongRow keeps one
  // marker entry with column -1 and is filtered by the CTA-per-row kernel).
  // Built when the padding stays below 30 % of the stored entries.
  bool sell = false;
  int64_t sell_len = 0;
  int64_t sell_cta_entries = 0;  // most entries in 8 consecutive slices (256 rows)
  flz::DevBuf<int32_t> sell_off;  // n_slices + 1 element offsets
  flz::DevBuf<int32_t> sell_col;
  flz::DevBuf<double> ssell64;
  flz::DevBuf<float> ssell32;
  flz::DevBuf<__nv_bfloat16> ssell16;
  flz::DevBuf<flz::dev::dfloat> sselldf;
  double ss_c[4] = {0.0, 0.0, 0.0, 0.0}, ss_e[4] = {0.0, 0.0, 0.0, 0.0};
  bool ss_ok[4] = {false, false, false, false};
  // Scratch of flz_filter_apply: recurrence vectors and the running sum.
  flz::DevBuf<double> ws64;
  flz::DevBuf<float> ws32;
  flz::DevBuf<__nv_bfloat16> ws16;
  flz::DevBuf<flz::dev::dfloat> wsdf;
  flz::FxValues fx;  // the fixed-point filter's values and scratch
  int32_t last_filter_precision = 0;  // flz_precision the last filter application ran in
};

// Solver handle: parameters, interval, results of the last solve and workspace.
struct flz_solver {
  flz_matrix* A = nullptr;
  flz_params p{};
  double alpha = 0.0, beta = 0.0;
  bool has_interval = false;
  bool solved = false;
  int64_t count = 0;
  std::vector<double> evals, resid;
  flz::DevBuf<double> evecs;  // n x count, column-major, ld = n
  flz_stats stats{};
  std::vector<flz_check> checks;  // the convergence checks of the last solve
  // workspace
  flz::DevBuf<double> Q, W, C, C2, part, X, AX, small, colpart;
  flz::TcBasis tcb;  // digit copy of the basis when reorthogonalization runs on the tensor cores
  // start vectors of the next solve (flz_solver_set_start_vectors): n x start_cols, column-major
  flz::DevBuf<double> start;
  int32_t start_cols = 0;
  double* pinned = nullptr;  // page-locked host words for the per-step D_j and S_j
  flz_solver() = default;
  flz_solver(const flz_solver&) = delete;
  flz_solver& operator=(const flz_solver&) = delete;
  ~flz_solver() {
    if (pinned) cudaFreeHost(pinned);
  }
};

namespace flz {

// Rows with more stored entries than this are filtered by one CTA each.
constexpr int kLongRow = 256;

// Block widths with a row-per-thread filter kernel (one thread owns a row and
// all its columns): powers of two with vector loads, and 3 (the paper's block
// size) element by element.
inline bool row_kernel_width(int r) { return r == 1 || r == 2 || r == 3 || r == 4 || r == 8 || r == 16; }
// Alignment a row-per-thread kernel needs of a block of `elem`-byte values.
inline size_t row_alignment(int r, size_t elem) {
  return (r & (r - 1)) ? elem : std::min<size_t>(16, (size_t)r * elem);
}

// ---- filter.cu ----------------------------------------------------------------
// W = p_m((A - cI)/e) V, V and W device FP64 n x r row-major.
void filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r,
                  const double* V, double* W, int precision, int recurrence, cudaStream_t st);
// The double-FP32 filter on blocks already stored as double-FP32 pairs (no
// conversion of V, W written as pairs).
void filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r,
                  const dev::dfloat* V, dev::dfloat* W, int recurrence, cudaStream_t st);
// ---- fixed.cu -------------------------------------------------------------------
// W = p_m(Ahat) V in 64-bit fixed point on the integer pipes (forward
// recurrence). Returns false, doing nothing, where the format does not apply
// (block width without a row kernel, a W not 16-byte aligned for even r, a
// row of 2 Ahat with absolute sum above 3.9, or coefficients too large):
// the caller then runs the FP64 filter. The overflow flag is fetched to the
// handle's host copy after the launches; read it with fx_check_flag after a
// synchronization of st.
bool fx_filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r, const double* V,
                     double* W, cudaStream_t st);
bool fx_supported(int r);
void fx_check_flag(flz_matrix* A);
// Batches. fx_batch_prepare builds the SELL-32 layout of the concatenation
// (once) and the fixed-point values of every problem's 2 Ahat_i = (2/e_i)(A_i -
// c_i I) (cc, ee: device arrays of c_i, e_i; d_off: the count + 1 row offsets);
// false where the fixed-point filter does not apply (padding above 30 %, rows
// longer than 256 entries, a shared-memory stage above its limit at width r,
// or a row of some 2 Ahat_i with absolute sum above 3.9): the batch then uses
// FP64. fx_batch_coefficients loads the per-problem coefficient tables
// (offset-binary, each problem's own sum scaling); false if a table does not
// fit the format. fx_batch_filter runs W = p_i(Ahat_i) Q_j for the active
// problems (j read from jdev on the device: graph-capturable); the columns of
// every problem's Q_j must have norm at most 1 (within 2^-20).
bool fx_batch_prepare(FxBatch& F, int64_t N, int64_t nnz, const int* rowptr, const int* col, const double* val,
                      const int* diag_pos, int32_t max_row_nnz, const int* d_off, const std::vector<int>& off_host,
                      int count, const double* cc, const double* ee, int r, cudaStream_t st);
bool fx_batch_coefficients(FxBatch& F, const std::vector<std::vector<double>>& coeffs, cudaStream_t st);
// persistent: every degree in one cooperative launch with a bounded grid
// barrier between degrees, instead of one launch per degree.
void fx_batch_filter(FxBatch& F, int r, const double* Q, const int* jdev, const int* d_off, const int* mdeg,
                     const int* active, double* W, bool pdl, bool persistent, cudaStream_t st);
// Reads and clears the batch filter's flag: FLZ_ERR_TIMEOUT (a stage wait
// expired) or FLZ_ERR_INVALID_ARG (a value left the format's range) raised.
void fx_batch_check_flag(FxBatch& F, cudaStream_t st);
// ---- refine.cu ---------------------------------------------------------------------
// Filtered subspace iteration in FP64-class arithmetic with Rayleigh-Ritz on A,
// polishing the pairs of a reduced-precision solve (see refine.cu).
struct RefineArgs {
  double alpha, beta, lmin, lmax, tol;
  int max_sweeps, max_degree;
  std::vector<double> filter;       // the solve's filter coefficients (interior windows)
  std::vector<double> filter_half;  // the same filter at half the degree (first sweep)
  int wanted;                       // pairs the reduced-precision solve found in the window
  // first sweep: the half-degree solve filter on the columns past `wanted`
  // only (the start vectors pass unchanged), whatever the window
  bool flat_first = false;
  // give up when a sweep does not halve the worst residual, or when the
  // products of A with a vector, extrapolated at the last sweep's rate to tol,
  // would pass matvec_budget (0: no budget)
  bool stop_on_stall = false;
  int64_t matvec_budget = 0;
  double range_scale = 1e-2;        // the damping polynomial's ratio across the window <= range_scale / residual
};
struct RefineResult {
  int sweeps = 0, kp = 0, filter_precision = 0;
  bool converged = false;
  std::vector<int> index;          // columns of X holding the wanted pairs
  std::vector<double> vals, res;   // their Rayleigh quotients and residuals / ||A||
  std::vector<int> degrees;        // filter degree of each sweep
  int64_t matvecs = 0;             // products of A with a vector in the filters (columns x degree)
  int outside = 0;                 // Ritz values of the final block outside [alpha, beta]
  double ms = 0.0;
};
// Device buffers of a refinement, kept across calls so that a caller refining
// many problems (one per host thread and stream) allocates and frees nothing
// per problem (cudaFree synchronizes the whole device).
struct RefineWorkspace {
  DevBuf<double> Y, AY, Vd, dev, part, S4, T4, Md, Hd;
  TcBasis tb;
};
// X: n x kp (kp a multiple of 16) as blocks of 16 columns, row-major; refined in place.
RefineResult refine(flz_matrix* A, const RefineArgs& g, double* X, int kp, cudaStream_t st,
                    RefineWorkspace* ws = nullptr);
// Chebyshev coefficients of T_d(a z + b) / T_d(-a + b), [zc, 1] mapped onto [-1, 1] by z -> a z + b.
void damping_coefficients(double zc, int d, double* out);
// ---- probe.cu ----------------------------------------------------------------------
// Measured throughput of FP64 FMAs (kind 0, flop/s) or 32-bit integer
// multiply-adds (kind 1, 2 ops each) on the current device.
double measure_alu_peak(int kind);
// ---- clenshaw.cu ----------------------------------------------------------------
// W = p_m(Ahat) V by the Clenshaw recurrence with 2 Ahat stored in `val`
// (MS; `vsell` in the SELL-32 layout or null, `val` in CSR order) and the
// recurrence vectors in VS; v is V in VS, ba and bb are n x r scratch, m >= 1.
template <class MS, class VS, class WT>
void run_clenshaw(const flz_matrix* A, const MS* vsell, const MS* val, const double* b, int m, int r, const VS* v,
                  VS* ba, VS* bb, WT* W, cudaStream_t st);
// Y = A X for an n x s block with row stride ld (s <= 16), FP64.
void spmm(const flz_matrix* A, const double* X, double* Y, int s, int ld, cudaStream_t st);

// ---- blockops.cu ------------------------------------------------------------------
// Basis layout: nb blocks, block b at Q + b * n * r, each n x r row-major.
// C[b][a][t] = sum_i Q_b[i, a] W[i, t] for t < s (W has row stride ldw), into
// device C (nb*r x s, row-major). `part` is scratch (see basis_dot_scratch).
size_t basis_dot_scratch(int64_t n, int nb, int r, int s);
void basis_dot(const double* Q, int nb, int64_t n, int r, const double* W, int s, int ldw, double* C,
               double* part, cudaStream_t st);
// The same with the basis and W stored as double-FP32 pairs and the products
// and sums formed on the FP32 pipes; C stays FP64.
void basis_dot(const dev::dfloat* Q, int nb, int64_t n, int r, const dev::dfloat* W, int s, int ldw, double* C,
               double* part, cudaStream_t st);
// Out[i, t] = beta * Out[i, t] + alpha * sum_{b, a} Q_b[i, a] C[(b*r + a)*s + t], t < s.
// Out has row stride ldo; Out may equal Q's block 0 when nb == 1 (in-place).
void basis_update(const double* Q, int nb, int64_t n, int r, const double* C, int s, double alpha,
                  double beta, double* Out, int ldo, cudaStream_t st);
void basis_update(const dev::dfloat* Q, int nb, int64_t n, int r, const double* C, int s, double alpha,
                  double beta, dev::dfloat* Out, int ldo, cudaStream_t st);
void basis_update(const dev::dfloat* Q, int nb, int64_t n, int r, const double* C, int s, double alpha,
                  double beta, double* Out, int ldo, cudaStream_t st);
// Per-column sums over rows: out[t] = sum_i X[i,t] Y[i,t] (mode 0) or
// sum_i (Y[i,t] - lam[t] X[i,t])^2 (mode 1); X, Y n x s with stride ld.
void column_sums(const double* X, const double* Y, const double* lam, int64_t n, int s, int ld, int mode,
                 double* out, double* part, cudaStream_t st);
size_t column_sums_scratch(int64_t n, int s);
// n x r block of N(0,1) numbers from a counter-based generator (seed, offset).
void random_normal(double* X, int64_t count, uint64_t seed, uint64_t offset, cudaStream_t st);
void random_normal(dev::dfloat* X, int64_t count, uint64_t seed, uint64_t offset, cudaStream_t st);
// Out = scale Out + X G: r combinations (G cols x r, row-major, device) of the
// cols columns of the column-major X (leading dimension ld) into the row-major
// n x r block Out.
void combine_columns(const double* X, int64_t n, int64_t ld, int cols, const double* G, int r, double scale,
                     double* Out, cudaStream_t st);
// Column j of a row-major n x s block (stride ld) into column-major out (stride ldo).
// out[t * ldo + i] = scale * X[i * ld + t] (row-major block to columns)
void rows_to_columns(const double* X, int64_t n, int s, int ld, double* out, int64_t ldo, cudaStream_t st,
                     double scale = 1.0);
// Block QR of the n x r block X (row-major) into Out (in place allowed) with
// no host round trip: CholeskyQR2, or shifted CholeskyQR3 when the first
// Cholesky factorization fails. scratch: qr_device_scratch() device doubles;
// on return S (the product of the factors, r x r upper triangular, X = Out S)
// is at scratch + 256.
size_t qr_device_scratch();
void qr_device(const double* X, double* Out, int64_t n, int r, double* scratch, cudaStream_t st);
// The inverse: column j of the column-major X (leading dimension ldx) into column
// j % 16 of the row-major 16-column block j / 16 of Out (blocks n * 16 apart).
void columns_to_blocks(const double* X, int64_t n, int64_t ldx, int cols, double* Out, cudaStream_t st);
// Gershgorin interval and max row length on the device.
void gershgorin(const flz_matrix* A, double* glo, double* ghi, int32_t* max_row_nnz);
// Structural/symmetry validation on the device; returns status (BAD_CSR, NOT_SYMMETRIC, OK).
flz_status validate_csr(const flz_matrix* A, int check_symmetry);
// Most stored entries in any `rows` consecutive rows starting at a multiple of `rows`.
int32_t max_block_nnz(const flz_matrix* A, int rows);
// Builds the SELL-32 structure of A (sell_off, sell_col) if its padding is
// below 30 % of the stored entries; sets A->sell.
void build_sell(flz_matrix* A);
// 2 Ahat = (2/e)(A - cI) in storage type S in the SELL-32 layout.
template <class S>
void scale_values_sell(const flz_matrix* A, double c, double e, S* out, cudaStream_t st);
// Fills A->diag_pos; returns the number of rows without a stored diagonal entry.
int64_t find_diagonals(flz_matrix* A);
// out[j] = (2/e)(val[j] - c [j is a diagonal position]) rounded to S.
template <class S>
void scale_values(const flz_matrix* A, double c, double e, S* out, cudaStream_t st);

// ---- hostla.cpp -------------------------------------------------------------------------
// Eigenvalues (ascending) of a symmetric band matrix (dense K x K storage,
// semi-bandwidth b): orthogonal band-to-tridiagonal reduction, then implicit QL.
void band_eigenvalues(const std::vector<double>& T, int K, int b, std::vector<double>& theta);
// Unit eigenvectors for the eigenvalues theta[idx[...]] by inverse iteration on
// the band matrix with partial pivoting; vectors of close eigenvalues are
// orthogonalized against each other. Y is K x count column-major.
void band_eigenvectors(const std::vector<double>& T, int K, int b, const std::vector<double>& theta,
                       const std::vector<int>& idx, std::vector<double>& Y, uint64_t seed,
                       const std::vector<double>* prevY = nullptr, const std::vector<int>* prevIdx = nullptr);
// Dense symmetric eigen-decomposition: A (n x n row-major, destroyed), w
// ascending, Z row-major with column k the eigenvector of w[k].
void dense_sym_eig(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& Z);
// Eigenvalues of a symmetric tridiagonal (d, e) by implicit QL; d overwritten ascending.
void tridiagonal_eigenvalues(std::vector<double>& d, std::vector<double>& e);
// Upper Cholesky factor R (G = R^T R) of an s x s SPD matrix, row-major; false if not SPD.
bool cholesky_upper(const double* G, int s, double* R);
// Inverse of an upper-triangular s x s matrix, row-major.
void upper_inverse(const double* R, int s, double* Rinv);

// ---- coefficients (api.cu) --------------------------------------------------------------
void chebyshev_coefficients(double a, double b, int m, double* out);
void smoothed_step_coefficients(double a, double b, double d, int m, double* out);
// The filter's coefficients for mapped [a, b]: the indicator's (Section 2.2)
// or, if transition > 0, the least-squares smoothed step's; then damping.
void filter_coeffs_for(const flz_params& p, double a, double b, int m, double* out);
void jackson_factors(int m, double* g);
void lanczos_sigma_factors(int m, double* g);
// Damping factors of params.damping (0: all ones, 1: Jackson, 2: Lanczos sigma).
void damping_factors(int damping, int m, double* g);
int auto_degree(double a, double b, double eps, int max_degree);

}  // namespace flz
