// Tall-skinny block kernels around the filter (Sections 2.3, 3.2.2):
//   basis_dot    C = Q^T W  over all basis blocks (full reorthogonalization,
//                Gram matrices of the block QR, D_j = Q_j^T p(A) Q_j)
//   basis_update Out = beta Out + alpha Q C (the projection update of
//                Gram-Schmidt, W R^{-1} of the block QR, Ritz vectors Q_k W_k)
//   column_sums  per-column dot products and residual norms (eq. rayleigh)
// plus the counter-based normal generator of the start blocks and CSR
// validation / Gershgorin bounds of the matrix handle.
//
// The basis is a sequence of n x r row-major blocks stored back to back, so
// a block is one contiguous slab and every kernel reads it with unit stride.
#include <algorithm>

#include "flz_internal.h"

namespace flz {

namespace {

constexpr int kThreads = 256;
// Rows of W staged in shared memory per sub-chunk, and the unrolling of the
// row loop: the FP64 form is bound by the FP64 pipe and keeps one row per
// lane in flight; the double-FP32 form is bound by memory latency and keeps
// four rows per lane (and twice the CTAs) in flight.
template <class T>
struct DotTune {
  static constexpr int kSub = 128, kRows = 1, kCtasPerSm = 4;
};
template <>
struct DotTune<dev::dfloat> {
  static constexpr int kSub = 256, kRows = 4, kCtasPerSm = 8;
};

using dev::dfloat;

// Arithmetic of the basis kernels: FP64, or double-FP32 pairs (hi + lo) on the
// FP32 pipes for a basis stored as dfloat (the FP64 rate is a small fraction
// of the FP32 rate on this GPU, and these kernels do r FMAs per loaded word).
template <class T>
__device__ __forceinline__ T zero_of();
template <>
__device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <>
__device__ __forceinline__ dfloat zero_of<dfloat>() { return dfloat(0.f, 0.f); }
__device__ __forceinline__ double ld_ro(const double* p) { return __ldg(p); }
__device__ __forceinline__ dfloat ld_ro(const dfloat* p) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(t.x, t.y);
}
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ dfloat shfl_down(dfloat v, int d) {
  return dfloat(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}
__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(dfloat x) { return dev::to_double(x); }
template <class T>
__device__ __forceinline__ T from_double(double x) { return T(x); }
template <class O, class A>
__device__ __forceinline__ O out_as(A x) { return x; }
template <>
__device__ __forceinline__ double out_as<double, dfloat>(dfloat x) { return dev::to_double(x); }

// Partial C = Q^T W over one row range (blockIdx.x) for a group of basis
// blocks (blockIdx.y). Warp w handles BPW blocks; lane l owns column
// a = l % R of rows l / R, l / R + 32/R, ... of the staged sub-chunk.
// T is the storage and arithmetic type of Q and W; partials are FP64.
template <int R, class T>
__global__ void __launch_bounds__(kThreads) basis_dot_kernel(const T* __restrict__ Q, int nb, long long n,
                                                             const T* __restrict__ W, int ldw,
                                                             long long rows_per_cta, double* __restrict__ part) {
  constexpr int BPW = (8 / R) > 0 ? (8 / R) : 1;
  constexpr int RPI = 32 / R;  // rows per warp iteration
  constexpr int kSub = DotTune<T>::kSub;
  constexpr int UR = DotTune<T>::kRows;
  __shared__ T wsm[kSub * R];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = lane % R, k = lane / R;
  const bool active = k < RPI;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  const int bbase = blockIdx.y * (8 * BPW) + warp * BPW;
  T acc[BPW][R];
#pragma unroll
  for (int bi = 0; bi < BPW; ++bi)
#pragma unroll
    for (int t = 0; t < R; ++t) acc[bi][t] = zero_of<T>();
  for (long long s0 = r0; s0 < r1; s0 += kSub) {
    const int rows = (int)min((long long)kSub, r1 - s0);
    for (int e = threadIdx.x; e < rows * R; e += kThreads) {
      const int i = e / R, t = e - i * R;
      wsm[e] = W[(size_t)(s0 + i) * ldw + t];
    }
    __syncthreads();
    if (active) {
      if constexpr (UR == 1) {
        // FP64: bound by the FP64 pipe; one row per lane per step
#pragma unroll
        for (int bi = 0; bi < BPW; ++bi) {
          const int b = bbase + bi;
          if (b < nb) {
            const T* qb = Q + (size_t)b * n * R + (size_t)s0 * R;
            for (int i = k; i < rows; i += RPI) {
              const T q = ld_ro(qb + (size_t)i * R + a);
#pragma unroll
              for (int t = 0; t < R; ++t) acc[bi][t] = fma(q, wsm[i * R + t], acc[bi][t]);
            }
          }
        }
      } else {
        // double-FP32: UR rows per lane and every block of the warp in flight before use
        int i = k;
        for (; i + (UR - 1) * RPI < rows; i += UR * RPI) {
          T q[BPW][UR];
#pragma unroll
          for (int bi = 0; bi < BPW; ++bi) {
            const T* qb = Q + (size_t)(bbase + bi) * n * R + (size_t)s0 * R;
#pragma unroll
            for (int u = 0; u < UR; ++u)
              q[bi][u] = (bbase + bi < nb) ? ld_ro(qb + (size_t)(i + u * RPI) * R + a) : zero_of<T>();
          }
#pragma unroll
          for (int bi = 0; bi < BPW; ++bi)
#pragma unroll
            for (int u = 0; u < UR; ++u)
#pragma unroll
              for (int t = 0; t < R; ++t) acc[bi][t] = fma(q[bi][u], wsm[(i + u * RPI) * R + t], acc[bi][t]);
        }
        for (; i < rows; i += RPI) {
#pragma unroll
          for (int bi = 0; bi < BPW; ++bi) {
            if (bbase + bi < nb) {
              const T q = ld_ro(Q + (size_t)(bbase + bi) * n * R + (size_t)(s0 + i) * R + a);
#pragma unroll
              for (int t = 0; t < R; ++t) acc[bi][t] = fma(q, wsm[i * R + t], acc[bi][t]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // reduce over the lanes sharing column a: lanes a, a+R, ..., a+(RPI-1)R
#pragma unroll
  for (int bi = 0; bi < BPW; ++bi) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      T v = acc[bi][t];
      for (int s = 1; s < RPI; s <<= 1) {
        const T o = shfl_down(v, s * R);
        if ((k & (2 * s - 1)) == 0 && k + s < RPI) v = v + o;
      }
      acc[bi][t] = v;
    }
  }
  if (k == 0) {
#pragma unroll
    for (int bi = 0; bi < BPW; ++bi) {
      const int b = bbase + bi;
      if (b < nb) {
        double* p = part + ((size_t)blockIdx.x * nb + b) * R * R + a * R;
#pragma unroll
        for (int t = 0; t < R; ++t) p[t] = as_double(acc[bi][t]);
      }
    }
  }
}

// out[o] = sum_p part[p][o]: 32 outputs per CTA, its 8 warps split the parts.
__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ part, int parts, size_t len,
                                                           double* __restrict__ out) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t o = (size_t)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (o < len)
    for (int p = w; p < parts; p += 8) s += part[(size_t)p * len + o];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && o < len) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) v += red[q][lane];
    out[o] = v;
  }
}

inline void sum_partials(const double* part, int parts, size_t len, double* out, cudaStream_t st) {
  sum_partials_kernel<<<(unsigned)((len + 31) / 32), 256, 0, st>>>(part, parts, len, out);
  FLZ_LAUNCH_CHECK();
}

// Out[i, t] = beta Out[i, t] + alpha sum_{b,a} Q_b[i, a] C[(b r + a) S + t], one thread per row.
// T: storage and arithmetic type of Q; O: storage type of Out; C is FP64.
template <int S, class T, class O>
__global__ void __launch_bounds__(kThreads) basis_update_kernel(const T* Q, int nb, long long n, int r,
                                                                const double* __restrict__ C, double alpha,
                                                                double beta, O* Out, int ldo) {
  extern __shared__ __align__(16) unsigned char csm_raw[];
  T* csm = reinterpret_cast<T*>(csm_raw);
  const int cb = max(1, 256 / r);  // basis blocks per staged chunk of C
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  T acc[S];
#pragma unroll
  for (int t = 0; t < S; ++t) acc[t] = zero_of<T>();
  for (int b0 = 0; b0 < nb; b0 += cb) {
    const int nbc = min(cb, nb - b0);
    __syncthreads();
    for (int e = threadIdx.x; e < nbc * r * S; e += kThreads) csm[e] = from_double<T>(C[(size_t)b0 * r * S + e]);
    __syncthreads();
    if (i < n) {
      for (int bl = 0; bl < nbc; ++bl) {
        const T* qrow = Q + (size_t)(b0 + bl) * n * r + (size_t)i * r;
        for (int a = 0; a < r; ++a) {
          const T q = qrow[a];
          const T* cr = csm + (bl * r + a) * S;
#pragma unroll
          for (int t = 0; t < S; ++t) acc[t] = fma(q, cr[t], acc[t]);
        }
      }
    }
  }
  if (i < n) {
    O* o = Out + (size_t)i * ldo;
    const T al = from_double<T>(alpha);
    if (beta == 0.0) {
#pragma unroll
      for (int t = 0; t < S; ++t) o[t] = out_as<O>(al * acc[t]);
    } else {
      const T be = from_double<T>(beta);
#pragma unroll
      for (int t = 0; t < S; ++t) {
        const T old = from_double<T>(as_double(o[t]));
        o[t] = out_as<O>(fma(al, acc[t], be * old));
      }
    }
  }
}

// Per-column sums over rows, s lanes per row; part[blockIdx.x][t].
__global__ void __launch_bounds__(kThreads) column_sums_kernel(const double* __restrict__ X,
                                                               const double* __restrict__ Y,
                                                               const double* __restrict__ lam, long long n, int s,
                                                               int ld, int mode, double* __restrict__ part) {
  __shared__ double red[kThreads];
  const int lane = threadIdx.x & 31;
  const int rpw = 32 / s;
  const int sub = lane / s, t = lane - sub * s;
  const long long warps_total = (long long)gridDim.x * (kThreads / 32);
  const long long warp = (long long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  double acc = 0.0;
  if (sub < rpw) {
    const double l = mode == 1 ? lam[t] : 0.0;
    for (long long row = warp * rpw + sub; row < n; row += warps_total * rpw) {
      const double x = X[(size_t)row * ld + t];
      const double y = Y[(size_t)row * ld + t];
      if (mode == 0) {
        acc = fma(x, y, acc);
      } else {
        const double d = y - l * x;
        acc = fma(d, d, acc);
      }
    }
  }
  red[threadIdx.x] = (sub < rpw) ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x < s) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w)
      for (int q = 0; q < rpw; ++q) v += red[w * 32 + q * s + threadIdx.x];
    part[(size_t)blockIdx.x * s + threadIdx.x] = v;
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// N(0,1) by Box-Muller on two counter-based uniforms (splitmix64 of seed and index).
template <class T>
__global__ void random_normal_kernel(T* __restrict__ X, long long count, uint64_t seed, uint64_t offset) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const uint64_t base = mix64(seed) ^ (2ull * (offset + (uint64_t)k));
    const double u1 = ((double)(mix64(base) >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
    const double u2 = (double)(mix64(base + 1) >> 11) * (1.0 / 9007199254740992.0);
    X[k] = from_double<T>(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
  }
}

__global__ void rows_to_columns_kernel(const double* __restrict__ X, long long n, int s, int ld,
                                       double* __restrict__ out, long long ldo, double scale) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * s;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / s;
    const int t = (int)(e - i * s);
    out[(size_t)t * ldo + i] = scale * X[(size_t)i * ld + t];
  }
}

__global__ void columns_to_blocks_kernel(const double* __restrict__ X, long long n, long long ldx, int cols,
                                         double* __restrict__ Out) {
  // one thread per (row, column) pair, consecutive threads along a row of a block
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * cols;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / (n * 16));
    const long long rem = e - (long long)b * n * 16;
    const int width = cols - 16 * b < 16 ? cols - 16 * b : 16;
    const long long i = rem / width;
    const int t = (int)(rem - i * width);
    Out[(size_t)b * n * 16 + (size_t)i * 16 + t] = X[(size_t)(16 * b + t) * ldx + i];
  }
}

__global__ void gershgorin_kernel(long long n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                  const double* __restrict__ val, double* __restrict__ lo, double* __restrict__ hi,
                                  int* __restrict__ maxlen) {
  __shared__ double slo[kThreads], shi[kThreads];
  __shared__ int slen[kThreads];
  double l = 1e308, h = -1e308;
  int len = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double d = 0.0, rad = 0.0;
    const int j0 = rowptr[i], j1 = rowptr[i + 1];
    for (int j = j0; j < j1; ++j) {
      if (col[j] == i) d += val[j];
      else rad += fabs(val[j]);
    }
    l = fmin(l, d - rad);
    h = fmax(h, d + rad);
    len = max(len, j1 - j0);
  }
  slo[threadIdx.x] = l;
  shi[threadIdx.x] = h;
  slen[threadIdx.x] = len;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
      slen[threadIdx.x] = max(slen[threadIdx.x], slen[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lo[blockIdx.x] = slo[0];
    hi[blockIdx.x] = shi[0];
    maxlen[blockIdx.x] = slen[0];
  }
}

// flags bit 0: structure error, bit 1: asymmetric value or missing transpose entry.
__global__ void validate_kernel(long long n, long long nnz, const int* __restrict__ rowptr,
                                const int* __restrict__ col, const double* __restrict__ val, int check_sym,
                                int* __restrict__ flags) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int j0 = rowptr[i], j1 = rowptr[i + 1];
    if ((i == 0 && j0 != 0) || j1 < j0 || (i == n - 1 && j1 != nnz) || j0 < 0 || j1 > nnz) {
      atomicOr(flags, 1);
      continue;
    }
    for (int j = j0; j < j1; ++j) {
      const int cj = col[j];
      if (cj < 0 || cj >= n || (j > j0 && col[j - 1] >= cj)) {
        atomicOr(flags, 1);
        break;
      }
      if (!check_sym) continue;
      // binary search for column i in row cj (row cj's structure may itself be
      // invalid; the search stays inside [rowptr[cj], rowptr[cj+1]) clipped to nnz)
      int lo = max(0, rowptr[cj]), hi = min((int)nnz, rowptr[cj + 1]) - 1;
      bool found = false;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = col[mid];
        if (cm == i) {
          const double x = val[j], y = val[mid];
          if (fabs(x - y) > 1e-14 * fmax(fabs(x), fabs(y))) atomicOr(flags, 2);
          found = true;
          break;
        }
        if (cm < i) lo = mid + 1;
        else hi = mid - 1;
      }
      if (!found) atomicOr(flags, 2);
    }
  }
}

// diag_pos[i] = index of column i within row i (binary search; columns are sorted), -1 if absent.
__global__ void find_diagonal_kernel(long long n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                     int* __restrict__ diag_pos, unsigned long long* __restrict__ missing) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int lo = rowptr[i], hi = rowptr[i + 1] - 1, pos = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int cm = col[mid];
      if (cm == i) {
        pos = mid;
        break;
      }
      if (cm < i) lo = mid + 1;
      else hi = mid - 1;
    }
    diag_pos[i] = pos;
    if (pos < 0) atomicAdd(missing, 1ull);
  }
}

template <class S>
__device__ __forceinline__ S round_to(double x);
template <>
__device__ __forceinline__ double round_to<double>(double x) { return x; }
template <>
__device__ __forceinline__ float round_to<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 round_to<__nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <>
__device__ __forceinline__ dev::dfloat round_to<dev::dfloat>(double x) { return dev::dfloat(x); }

template <class S>
__global__ void scale_values_kernel(long long n, const int* __restrict__ rowptr, const int* __restrict__ diag_pos,
                                    const double* __restrict__ val, double s, double shift, S* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int d = diag_pos[i];
    for (int j = rowptr[i], je = rowptr[i + 1]; j < je; ++j) out[j] = round_to<S>(s * (val[j] - (j == d ? shift : 0.0)));
  }
}

inline unsigned gs_blocks(long long count) {
  return (unsigned)std::max<long long>(1, std::min<long long>((count + 255) / 256, 152 * 16));
}

struct DotShape {
  int gx, gy;
  long long rows_per_cta;
};

template <class T>
DotShape dot_shape(int64_t n, int nb, int r) {
  constexpr int kSub = DotTune<T>::kSub;
  const int bpw = std::max(1, 8 / r);
  const int bpc = 8 * bpw;
  DotShape d;
  d.gy = (nb + bpc - 1) / bpc;
  const long long max_gx = std::max<long long>(1, (n + kSub - 1) / kSub);
  d.gx = (int)std::min<long long>(max_gx, std::max(1, DotTune<T>::kCtasPerSm * 152 / d.gy));
  d.rows_per_cta = ((n + d.gx - 1) / d.gx + kSub - 1) / kSub * kSub;
  d.gx = (int)((n + d.rows_per_cta - 1) / d.rows_per_cta);
  return d;
}

template <int R, class T>
void launch_basis_dot(const T* Q, int nb, int64_t n, const T* W, int ldw, double* C, double* part, cudaStream_t st) {
  const DotShape d = dot_shape<T>(n, nb, R);
  basis_dot_kernel<R, T><<<dim3(d.gx, d.gy), kThreads, 0, st>>>(Q, nb, n, W, ldw, d.rows_per_cta, part);
  FLZ_LAUNCH_CHECK();
  sum_partials(part, d.gx, (size_t)nb * R * R, C, st);
}

template <int S, class T, class O>
void launch_basis_update(const T* Q, int nb, int64_t n, int r, const double* C, double alpha, double beta, O* Out,
                         int ldo, cudaStream_t st) {
  const int cb = std::max(1, 256 / r);
  const size_t smem = sizeof(T) * (size_t)std::min(cb, nb) * r * S;
  if (smem > 48 * 1024)
    FLZ_CUDA(cudaFuncSetAttribute(basis_update_kernel<S, T, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
  basis_update_kernel<S, T, O><<<grid, kThreads, smem, st>>>(Q, nb, n, r, C, alpha, beta, Out, ldo);
  FLZ_LAUNCH_CHECK();
}

}  // namespace

size_t basis_dot_scratch(int64_t n, int nb, int r, int s) {
  (void)s;
  // the largest partial-sum buffer any call with 1..nb blocks needs
  size_t best = 0;
  for (int b = 1; b <= nb; ++b) {
    const DotShape d = dot_shape<double>(n, b, r);
    const DotShape e = dot_shape<dev::dfloat>(n, b, r);
    best = std::max(best, (size_t)std::max(d.gx, e.gx) * b * r * r);
  }
  return best;
}

// Runs STMT with the compile-time width K = X (1..16).
#define FLZ_WITH_WIDTH(X, STMT) \
  switch (X) { \
    case 1: { constexpr int K = 1; STMT; } break; \
    case 2: { constexpr int K = 2; STMT; } break; \
    case 3: { constexpr int K = 3; STMT; } break; \
    case 4: { constexpr int K = 4; STMT; } break; \
    case 5: { constexpr int K = 5; STMT; } break; \
    case 6: { constexpr int K = 6; STMT; } break; \
    case 7: { constexpr int K = 7; STMT; } break; \
    case 8: { constexpr int K = 8; STMT; } break; \
    case 9: { constexpr int K = 9; STMT; } break; \
    case 10: { constexpr int K = 10; STMT; } break; \
    case 11: { constexpr int K = 11; STMT; } break; \
    case 12: { constexpr int K = 12; STMT; } break; \
    case 13: { constexpr int K = 13; STMT; } break; \
    case 14: { constexpr int K = 14; STMT; } break; \
    case 15: { constexpr int K = 15; STMT; } break; \
    case 16: { constexpr int K = 16; STMT; } break; \
    default: fail(FLZ_ERR_INVALID_ARG, "block width %d out of range 1..16", (int)(X)); \
  }

namespace {

template <class T>
void basis_dot_t(const T* Q, int nb, int64_t n, int r, const T* W, int s, int ldw, double* C, double* part,
                 cudaStream_t st) {
  if (s != r) fail(FLZ_ERR_INVALID_ARG, "basis_dot needs s == r");
  if (nb <= 0) return;
  FLZ_WITH_WIDTH(r, (launch_basis_dot<K, T>(Q, nb, n, W, ldw, C, part, st)));
}

template <class T, class O>
void basis_update_t(const T* Q, int nb, int64_t n, int r, const double* C, int s, double alpha, double beta, O* Out,
                    int ldo, cudaStream_t st) {
  if (nb <= 0) return;
  FLZ_WITH_WIDTH(s, (launch_basis_update<K, T, O>(Q, nb, n, r, C, alpha, beta, Out, ldo, st)));
}

}  // namespace

void basis_dot(const double* Q, int nb, int64_t n, int r, const double* W, int s, int ldw, double* C,
               double* part, cudaStream_t st) {
  basis_dot_t<double>(Q, nb, n, r, W, s, ldw, C, part, st);
}
void basis_dot(const dfloat* Q, int nb, int64_t n, int r, const dfloat* W, int s, int ldw, double* C,
               double* part, cudaStream_t st) {
  basis_dot_t<dfloat>(Q, nb, n, r, W, s, ldw, C, part, st);
}

void basis_update(const double* Q, int nb, int64_t n, int r, const double* C, int s, double alpha, double beta,
                  double* Out, int ldo, cudaStream_t st) {
  basis_update_t<double, double>(Q, nb, n, r, C, s, alpha, beta, Out, ldo, st);
}
void basis_update(const dfloat* Q, int nb, int64_t n, int r, const double* C, int s, double alpha, double beta,
                  dfloat* Out, int ldo, cudaStream_t st) {
  basis_update_t<dfloat, dfloat>(Q, nb, n, r, C, s, alpha, beta, Out, ldo, st);
}
void basis_update(const dfloat* Q, int nb, int64_t n, int r, const double* C, int s, double alpha, double beta,
                  double* Out, int ldo, cudaStream_t st) {
  basis_update_t<dfloat, double>(Q, nb, n, r, C, s, alpha, beta, Out, ldo, st);
}

size_t column_sums_scratch(int64_t n, int s) {
  (void)n;
  return (size_t)152 * 4 * s;
}

void column_sums(const double* X, const double* Y, const double* lam, int64_t n, int s, int ld, int mode,
                 double* out, double* part, cudaStream_t st) {
  const int rpw = 32 / s;
  const long long warps = (n + rpw - 1) / rpw;
  const int grid = (int)std::max<long long>(1, std::min<long long>(152 * 4, (warps + 7) / 8));
  column_sums_kernel<<<grid, kThreads, 0, st>>>(X, Y, lam, n, s, ld, mode, part);
  FLZ_LAUNCH_CHECK();
  sum_partials(part, grid, (size_t)s, out, st);
}

// Out[i, t] = scale * Out[i, t] + sum_j X[i + j ld] G[j r + t] for t < r: r
// combinations of the `cols` columns of the column-major X added to a
// (row-major) n x r block. One thread per row; X read with unit stride
// across the threads of a warp.
template <int R>
__global__ void combine_columns_kernel(const double* __restrict__ X, long long n, long long ld, int cols,
                                       const double* __restrict__ G, double scale, double* __restrict__ Out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc[R];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = scale * Out[i * R + t];
    for (int j = 0; j < cols; ++j) {
      const double x = X[(size_t)j * ld + i];
#pragma unroll
      for (int t = 0; t < R; ++t) acc[t] = fma(x, __ldg(G + j * R + t), acc[t]);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) Out[i * R + t] = acc[t];
  }
}

void combine_columns(const double* X, int64_t n, int64_t ld, int cols, const double* G, int r, double scale,
                     double* Out, cudaStream_t st) {
  const unsigned grid = gs_blocks(n);
  switch (r) {
#define FLZ_CC(R)                                                                                      \
  case R:                                                                                              \
    combine_columns_kernel<R><<<grid, 256, 0, st>>>(X, n, ld, cols, G, scale, Out); \
    break;
    FLZ_CC(1) FLZ_CC(2) FLZ_CC(3) FLZ_CC(4) FLZ_CC(5) FLZ_CC(6) FLZ_CC(7) FLZ_CC(8)
    FLZ_CC(9) FLZ_CC(10) FLZ_CC(11) FLZ_CC(12) FLZ_CC(13) FLZ_CC(14) FLZ_CC(15) FLZ_CC(16)
#undef FLZ_CC
    default: fail(FLZ_ERR_INVALID_ARG, "block width %d", r);
  }
  FLZ_LAUNCH_CHECK();
}

void random_normal(double* X, int64_t count, uint64_t seed, uint64_t offset, cudaStream_t st) {
  random_normal_kernel<double><<<gs_blocks(count), 256, 0, st>>>(X, count, seed, offset);
  FLZ_LAUNCH_CHECK();
}
void random_normal(dfloat* X, int64_t count, uint64_t seed, uint64_t offset, cudaStream_t st) {
  random_normal_kernel<dfloat><<<gs_blocks(count), 256, 0, st>>>(X, count, seed, offset);
  FLZ_LAUNCH_CHECK();
}

void rows_to_columns(const double* X, int64_t n, int s, int ld, double* out, int64_t ldo, cudaStream_t st,
                     double scale) {
  rows_to_columns_kernel<<<gs_blocks(n * s), 256, 0, st>>>(X, n, s, ld, out, ldo, scale);
  FLZ_LAUNCH_CHECK();
}

// ---- device CholeskyQR (single solver) ----------------------------------------
// Passes X -> X R_1^{-1} -> ... of an n x R block, every small step on the
// device. A pass: the Gram matrix's upper triangle as per-CTA partial sums
// (R(R+1)/2 products per row, not R^2), its factorization, and the
// triangular update (R(R+1)/2 products per row). The third pass runs only if
// the first needed the shift (shifted CholeskyQR3; otherwise CholeskyQR2):
// its kernels read the skip word the first factorization wrote.
constexpr int kQrParts = 152 * 2;

template <int R>
__global__ void __launch_bounds__(kThreads) qr_gram_kernel(const double* __restrict__ X, long long n,
                                                           double* __restrict__ part, const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int NT = R * (R + 1) / 2;
  double g[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) g[t] = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    double x[R];
#pragma unroll
    for (int a = 0; a < R; ++a) x[a] = X[i * R + a];
    int t = 0;
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = a; b < R; ++b) {
        g[t] = fma(x[a], x[b], g[t]);
        ++t;
      }
  }
  __shared__ double red[kThreads / 32][NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    double v = g[t];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NT; t += kThreads) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][t];
    part[(size_t)blockIdx.x * NT + t] = v;
  }
}

// Sums the partial Gram triangles (fixed order), then on one thread: R with
// R^T R = G; on pass 0 a failed factorization is retried with G + shift I,
// shift = 11 (n r + r (r + 1)) u max_i G_ii r, and skip[0] records whether the
// third pass can be skipped; a factorization that still fails keeps
// R = diag(sqrt(G_ii)). Rinv = R^{-1}, S = R S (S = R on pass 0).
__global__ void qr_factor_kernel(const double* __restrict__ part, int nparts, int r, double nrows, int pass,
                                 double* __restrict__ Rinv, double* __restrict__ S, int* __restrict__ skip) {
  if (pass == 2 && *skip) return;
  const int NT = r * (r + 1) / 2;
  __shared__ double gs[16 * 17 / 2];
  // entry t of the triangle summed by one warp (lanes over the partial
  // sums, then a fixed shuffle tree: the same order on every run)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = warp; t < NT; t += nw) {
    double v = 0.0;
    for (int q = lane; q < nparts; q += 32) v += part[(size_t)q * NT + t];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) gs[t] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double G[16 * 16], R[16 * 16], Ri[16 * 16];
  for (int a = 0, t = 0; a < r; ++a)
    for (int b = a; b < r; ++b, ++t) G[a * r + b] = G[b * r + a] = gs[t];
  auto factor = [&](double shift) {
    for (int a = 0; a < r * r; ++a) R[a] = 0.0;
    for (int a = 0; a < r; ++a) {
      double d = G[a * r + a] + shift;
      for (int q = 0; q < a; ++q) d -= R[q * r + a] * R[q * r + a];
      if (!(d > 0.0)) return false;
      const double rd = sqrt(d);
      R[a * r + a] = rd;
      for (int b = a + 1; b < r; ++b) {
        double v = G[a * r + b];
        for (int q = 0; q < a; ++q) v -= R[q * r + a] * R[q * r + b];
        R[a * r + b] = v / rd;
      }
    }
    return true;
  };
  bool ok = factor(0.0);
  if (pass == 0) *skip = ok ? 1 : 0;
  if (!ok && pass == 0) {
    double gmax = 0.0;
    for (int d = 0; d < r; ++d) gmax = fmax(gmax, G[d * r + d]);
    ok = factor(11.0 * (nrows * r + (double)r * (r + 1)) * 1.1102230246251565e-16 * fmax(gmax * r, 1e-300));
  }
  if (!ok) {
    for (int a = 0; a < r * r; ++a) R[a] = 0.0;
    for (int a = 0; a < r; ++a) R[a * r + a] = sqrt(fmax(G[a * r + a], 1e-300));
  }
  for (int a = 0; a < r * r; ++a) Ri[a] = 0.0;
  for (int b = 0; b < r; ++b) {
    Ri[b * r + b] = 1.0 / R[b * r + b];
    for (int a = b - 1; a >= 0; --a) {
      double v = 0.0;
      for (int q = a + 1; q <= b; ++q) v += R[a * r + q] * Ri[q * r + b];
      Ri[a * r + b] = -v / R[a * r + a];
    }
  }
  for (int a = 0; a < r * r; ++a) Rinv[a] = Ri[a];
  if (pass == 0) {
    for (int a = 0; a < r * r; ++a) S[a] = R[a];
  } else {
    double T[16 * 16];
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) {
        double v = 0.0;
        for (int q = 0; q < r; ++q) v += R[a * r + q] * S[q * r + b];
        T[a * r + b] = v;
      }
    for (int a = 0; a < r * r; ++a) S[a] = T[a];
  }
}

// Out = X Rinv with Rinv upper triangular (in place allowed: a row is read whole first)
template <int R>
__global__ void __launch_bounds__(kThreads) qr_update_kernel(const double* X, const double* __restrict__ Rinv,
                                                             double* Out, long long n, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double ri[R * R];
  for (int t = threadIdx.x; t < R * R; t += kThreads) ri[t] = Rinv[t];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    double x[R], y[R];
#pragma unroll
    for (int a = 0; a < R; ++a) x[a] = X[i * R + a];
#pragma unroll
    for (int b = 0; b < R; ++b) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a <= b; ++a) v = fma(x[a], ri[a * R + b], v);
      y[b] = v;
    }
#pragma unroll
    for (int b = 0; b < R; ++b) Out[i * R + b] = y[b];
  }
}

template <int R>
void qr_device_r(const double* X, double* Out, int64_t n, double* scratch, cudaStream_t st) {
  double* Rinv = scratch;
  double* S = scratch + 256;
  int* skip = reinterpret_cast<int*>(scratch + 512);
  double* part = scratch + 520;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(kQrParts, (n + kThreads - 1) / kThreads));
  const double* src = X;
  for (int pass = 0; pass < 3; ++pass) {
    const int* sk = pass == 2 ? skip : nullptr;
    qr_gram_kernel<R><<<grid, kThreads, 0, st>>>(src, n, part, sk);
    FLZ_LAUNCH_CHECK();
    qr_factor_kernel<<<1, 256, 0, st>>>(part, (int)grid, R, (double)n, pass, Rinv, S, skip);
    FLZ_LAUNCH_CHECK();
    qr_update_kernel<R><<<gs_blocks(n), kThreads, 0, st>>>(src, Rinv, Out, n, sk);
    FLZ_LAUNCH_CHECK();
    src = Out;
  }
}

size_t qr_device_scratch() { return 520 + (size_t)kQrParts * 136; }

void qr_device(const double* X, double* Out, int64_t n, int r, double* scratch, cudaStream_t st) {
  switch (r) {
#define FLZ_QR(R_) \
  case R_:         \
    qr_device_r<R_>(X, Out, n, scratch, st); \
    break;
    FLZ_QR(1) FLZ_QR(2) FLZ_QR(3) FLZ_QR(4) FLZ_QR(5) FLZ_QR(6) FLZ_QR(7) FLZ_QR(8)
    FLZ_QR(9) FLZ_QR(10) FLZ_QR(11) FLZ_QR(12) FLZ_QR(13) FLZ_QR(14) FLZ_QR(15) FLZ_QR(16)
#undef FLZ_QR
    default: fail(FLZ_ERR_INVALID_ARG, "block width %d", r);
  }
}

void columns_to_blocks(const double* X, int64_t n, int64_t ldx, int cols, double* Out, cudaStream_t st) {
  if (cols <= 0 || n <= 0) return;
  columns_to_blocks_kernel<<<gs_blocks(n * cols), 256, 0, st>>>(X, n, ldx, cols, Out);
  FLZ_LAUNCH_CHECK();
}

void gershgorin(const flz_matrix* A, double* glo, double* ghi, int32_t* max_row_nnz) {
  const unsigned grid = gs_blocks(A->n);
  DevBuf<double> lo, hi;
  DevBuf<int> len;
  lo.reserve(grid);
  hi.reserve(grid);
  len.reserve(grid);
  gershgorin_kernel<<<grid, kThreads>>>(A->n, A->rowptr.p, A->col.p, A->val.p, lo.p, hi.p, len.p);
  FLZ_LAUNCH_CHECK();
  std::vector<double> hlo(grid), hhi(grid);
  std::vector<int> hlen(grid);
  FLZ_CUDA(cudaMemcpy(hlo.data(), lo.p, grid * sizeof(double), cudaMemcpyDeviceToHost));
  FLZ_CUDA(cudaMemcpy(hhi.data(), hi.p, grid * sizeof(double), cudaMemcpyDeviceToHost));
  FLZ_CUDA(cudaMemcpy(hlen.data(), len.p, grid * sizeof(int), cudaMemcpyDeviceToHost));
  *glo = *std::min_element(hlo.begin(), hlo.end());
  *ghi = *std::max_element(hhi.begin(), hhi.end());
  *max_row_nnz = *std::max_element(hlen.begin(), hlen.end());
}

__global__ void block_nnz_kernel(long long n, int rows, const int* __restrict__ rowptr, int* __restrict__ best) {
  const long long nblk = (n + rows - 1) / rows;
  for (long long bk = (long long)blockIdx.x * blockDim.x + threadIdx.x; bk < nblk; bk += (long long)gridDim.x * blockDim.x) {
    const long long r0 = bk * rows, r1 = min(n, r0 + rows);
    atomicMax(best, rowptr[r1] - rowptr[r0]);
  }
}

int32_t max_block_nnz(const flz_matrix* A, int rows) {
  DevBuf<int> best;
  best.reserve(1);
  FLZ_CUDA(cudaMemset(best.p, 0, sizeof(int)));
  block_nnz_kernel<<<gs_blocks((A->n + rows - 1) / rows), 256>>>(A->n, rows, A->rowptr.p, best.p);
  FLZ_LAUNCH_CHECK();
  int h = 0;
  FLZ_CUDA(cudaMemcpy(&h, best.p, sizeof(int), cudaMemcpyDeviceToHost));
  return h;
}

// Slice widths of the SELL-32 layout: the longest row of each 32-row slice,
// counting a row longer than `long_row` as one marker entry.
__global__ void sell_width_kernel(long long n, const int* __restrict__ rowptr, int long_row, int* __restrict__ width) {
  const long long nsl = (n + 31) / 32;
  for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < nsl; sl += (long long)gridDim.x * blockDim.x) {
    int w = 1;
    for (long long i = sl * 32; i < min(n, sl * 32 + 32); ++i) {
      const int len = rowptr[i + 1] - rowptr[i];
      w = max(w, len > long_row ? 1 : len);
    }
    width[sl] = w;
  }
}

// SELL-32 columns: a row's entries in order, then padding with its own index;
// a long row gets the marker -1 in its first slot.
__global__ void sell_fill_col_kernel(long long n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                     int long_row, const int* __restrict__ off, int* __restrict__ scol) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long sl = i >> 5;
    const int lane = (int)(i & 31);
    const int base = off[sl] + lane;
    const int w = (off[sl + 1] - off[sl]) >> 5;
    const int j0 = rowptr[i], len = rowptr[i + 1] - j0;
    const bool is_long = len > long_row;
    for (int j = 0; j < w; ++j) {
      int c = (int)i;
      if (is_long) c = j == 0 ? -1 : (int)i;
      else if (j < len) c = col[j0 + j];
      scol[base + 32 * j] = c;
    }
  }
}

template <class S>
__global__ void scale_values_sell_kernel(long long n, const int* __restrict__ rowptr, const int* __restrict__ diag_pos,
                                         const double* __restrict__ val, int long_row, const int* __restrict__ off,
                                         double s, double shift, S* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long sl = i >> 5;
    const int lane = (int)(i & 31);
    const int base = off[sl] + lane;
    const int w = (off[sl + 1] - off[sl]) >> 5;
    const int j0 = rowptr[i], len = rowptr[i + 1] - j0;
    const int d = diag_pos[i];
    for (int j = 0; j < w; ++j) {
      double v = 0.0;
      if (len <= long_row && j < len) v = s * (val[j0 + j] - (j0 + j == d ? shift : 0.0));
      out[base + 32 * j] = round_to<S>(v);
    }
  }
}

void build_sell(flz_matrix* A) {
  A->sell = false;
  const int64_t nsl = (A->n + 31) / 32;
  DevBuf<int> width;
  width.reserve((size_t)nsl);
  sell_width_kernel<<<gs_blocks(nsl), 256>>>(A->n, A->rowptr.p, kLongRow, width.p);
  FLZ_LAUNCH_CHECK();
  std::vector<int> hw(nsl);
  FLZ_CUDA(cudaMemcpy(hw.data(), width.p, sizeof(int) * nsl, cudaMemcpyDeviceToHost));
  std::vector<int32_t> off(nsl + 1);
  int64_t total = 0;
  for (int64_t sl = 0; sl < nsl; ++sl) {
    off[sl] = (int32_t)std::min<int64_t>(total, 0x7fffffff);
    total += 32 * (int64_t)hw[sl];
  }
  off[nsl] = (int32_t)std::min<int64_t>(total, 0x7fffffff);
  // worthwhile only when the padding is small (regular stencils, not power-law graphs)
  if (total >= 0x7fffffff || (double)total > 1.3 * (double)std::max<int64_t>(A->nnz, 1)) return;
  A->sell_off.reserve((size_t)nsl + 1);
  FLZ_CUDA(cudaMemcpy(A->sell_off.p, off.data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice));
  A->sell_col.reserve((size_t)std::max<int64_t>(total, 1));
  sell_fill_col_kernel<<<gs_blocks(A->n), 256>>>(A->n, A->rowptr.p, A->col.p, kLongRow, A->sell_off.p, A->sell_col.p);
  FLZ_LAUNCH_CHECK();
  FLZ_CUDA(cudaDeviceSynchronize());
  A->sell_len = total;
  // the most entries any CTA of 256 rows (8 slices) holds: the shared-memory
  // stage of the staged SELL kernels
  int64_t cta_max = 0;
  for (int64_t s0 = 0; s0 < nsl; s0 += 8) cta_max = std::max<int64_t>(cta_max, off[std::min(nsl, s0 + 8)] - off[s0]);
  A->sell_cta_entries = cta_max;
  A->sell = true;
}

template <class S>
void scale_values_sell(const flz_matrix* A, double c, double e, S* out, cudaStream_t st) {
  scale_values_sell_kernel<S><<<gs_blocks(A->n), 256, 0, st>>>(A->n, A->rowptr.p, A->diag_pos.p, A->val.p, kLongRow,
                                                               A->sell_off.p, 2.0 / e, c, out);
  FLZ_LAUNCH_CHECK();
}
template void scale_values_sell<double>(const flz_matrix*, double, double, double*, cudaStream_t);
template void scale_values_sell<float>(const flz_matrix*, double, double, float*, cudaStream_t);
template void scale_values_sell<__nv_bfloat16>(const flz_matrix*, double, double, __nv_bfloat16*, cudaStream_t);
template void scale_values_sell<dev::dfloat>(const flz_matrix*, double, double, dev::dfloat*, cudaStream_t);

int64_t find_diagonals(flz_matrix* A) {
  A->diag_pos.reserve((size_t)A->n);
  DevBuf<unsigned long long> missing;
  missing.reserve(1);
  FLZ_CUDA(cudaMemset(missing.p, 0, sizeof(unsigned long long)));
  find_diagonal_kernel<<<gs_blocks(A->n), 256>>>(A->n, A->rowptr.p, A->col.p, A->diag_pos.p, missing.p);
  FLZ_LAUNCH_CHECK();
  unsigned long long h = 0;
  FLZ_CUDA(cudaMemcpy(&h, missing.p, sizeof(h), cudaMemcpyDeviceToHost));
  return (int64_t)h;
}

template <class S>
void scale_values(const flz_matrix* A, double c, double e, S* out, cudaStream_t st) {
  scale_values_kernel<S><<<gs_blocks(A->n), 256, 0, st>>>(A->n, A->rowptr.p, A->diag_pos.p, A->val.p, 2.0 / e, c, out);
  FLZ_LAUNCH_CHECK();
}
template void scale_values<double>(const flz_matrix*, double, double, double*, cudaStream_t);
template void scale_values<float>(const flz_matrix*, double, double, float*, cudaStream_t);
template void scale_values<__nv_bfloat16>(const flz_matrix*, double, double, __nv_bfloat16*, cudaStream_t);
template void scale_values<dev::dfloat>(const flz_matrix*, double, double, dev::dfloat*, cudaStream_t);

flz_status validate_csr(const flz_matrix* A, int check_symmetry) {
  DevBuf<int> flags;
  flags.reserve(1);
  FLZ_CUDA(cudaMemset(flags.p, 0, sizeof(int)));
  validate_kernel<<<gs_blocks(A->n), 256>>>(A->n, A->nnz, A->rowptr.p, A->col.p, A->val.p, check_symmetry,
                                            flags.p);
  FLZ_LAUNCH_CHECK();
  int h = 0;
  FLZ_CUDA(cudaMemcpy(&h, flags.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h & 1) return FLZ_ERR_BAD_CSR;
  if (h & 2) return FLZ_ERR_NOT_SYMMETRIC;
  return FLZ_OK;
}

}  // namespace flz
