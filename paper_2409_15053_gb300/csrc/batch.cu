// Batches of independent filtered Lanczos problems, solved in lockstep.
//
// The paper solves one matrix per call (Section 3.2). Here `count` problems
// (matrix, interval) share every kernel launch: their CSR matrices are
// concatenated into one block-diagonal device matrix, block vectors are
// concatenated row-wise, and each kernel finds the problem of a row from the
// row offsets. Per problem: spectrum bounds, map (eq. transf), degree
// (eq. optimaldegree) and coefficients (Section 2.2); segmented
// reductions give each problem its own Q^T W, Gram matrices and block QR; the
// convergence test (Section 3.2.2) runs per problem on the host. A problem
// that converges is masked out of all later work.
//
// Everything between two checks is device-resident: the step index lives in
// device memory and the block QR factors are computed on the device, so one
// whole block Lanczos step (filter degrees, CGS2, shifted CholeskyQR3,
// history of D_j and S_j) is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <thread>
#include <atomic>
#include <string>

#include "device_common.cuh"
#include "flz_internal.h"

struct flz_batch {
  int count = 0;
  std::vector<flz_matrix*> mats;
  std::vector<double> alpha, beta;
  flz_params p{};
  int r = 0;  // block width in use
  // block-diagonal concatenation
  int64_t N = 0, nnz = 0;
  std::vector<int> off;  // count + 1 row offsets
  flz::DevBuf<int> d_off, rowptr, col, diag_pos;
  flz::DevBuf<double> val;
  int max_cta_nnz = 0;
  // chunks of rows (never straddling two problems) for segmented reductions
  std::vector<int> c_row0, c_row1, c_mat, c_beg;
  flz::DevBuf<int> d_c_row0, d_c_row1, d_c_mat, d_c_beg;
  // results
  bool solved = false;
  std::vector<std::vector<double>> evals, resid;
  std::vector<std::unique_ptr<flz::DevBuf<double>>> evecs;  // n_i x count_i column-major
  std::vector<flz_stats> stats;
  int32_t max_row_nnz = 0;  // longest row of any problem
  flz::FxBatch fxb;         // the fixed-point filter's layout and tables
  int tuned_r = 0, tuned_rows = 0;  // the autotuner's choices, kept for the handle's later solves
};

namespace flz {

using namespace dev;

namespace {

constexpr int kT = 256;
constexpr int kRowsB = 256;
constexpr int kSubB = 128;
constexpr int kMaxProblems = 4096;

// Problem of `row`: the largest i with off[i] <= row (off in shared memory).
__device__ __forceinline__ int problem_of(const int* soff, int count, int row) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (soff[mid] <= row) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Fused degree step over all problems (same arithmetic as the single-problem
// kernel) with per-problem coefficients coef[k * count + i] and degrees.
template <int R, class MS, class VS, class AccS, bool FIRST>
__global__ void __launch_bounds__(kRowsB) seg_cheb_kernel(
    int N, int cap, const int* __restrict__ rowptr, const int* __restrict__ col, const MS* __restrict__ sval,
    const int* __restrict__ off, int count, const double* __restrict__ coef, int k, const int* __restrict__ mdeg,
    const int* __restrict__ active, const VS* __restrict__ ycur, const VS* yprev, VS* ynext, AccS* acc_io) {
  using A = typename Arith<VS>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  MS* s_val = reinterpret_cast<MS*>(smem);
  int* s_col = reinterpret_cast<int*>(smem + (size_t)cap * sizeof(MS));
  int* s_off = s_col + cap;
  for (int i = threadIdx.x; i <= count; i += kRowsB) s_off[i] = off[i];
  const int row0 = blockIdx.x * kRowsB;
  const int rend = min(N, row0 + kRowsB);
  const int row = row0 + (int)threadIdx.x;
  const int j0 = __ldg(rowptr + row0);
  const int j1 = __ldg(rowptr + rend);
  const bool staged = (j1 - j0) <= cap;
  if (staged) {
    for (int e = threadIdx.x; e < j1 - j0; e += kRowsB) {
      s_col[e] = __ldg(col + j0 + e);
      s_val[e] = sval[j0 + e];
    }
  }
  __syncthreads();
  allow_dependents();
  if (row >= N) return;
  const int pi = problem_of(s_off, count, row);
  if (!active[pi] || k + 1 > mdeg[pi]) return;
  const int jb = __ldg(rowptr + row), je = __ldg(rowptr + row + 1);
  grid_dependency_wait();  // the vectors below are the previous degree's output
  A s[R];
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = A(0);
  } else {
    load_row<VS, R>(yprev + (size_t)row * R, s);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = -s[t];
  }
  // U independent row gathers in flight per thread (fewer for wide rows)
  constexpr int kRowBytes = R * (int)sizeof(A);
  constexpr int U = kRowBytes <= 16 ? 4 : (kRowBytes <= 32 ? 2 : 1);
  int j = jb;
  for (; j + U <= je; j += U) {
    int cj[U];
    A a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cj[u] = staged ? s_col[j + u - j0] : __ldg(col + j + u);
      a[u] = staged ? to_arith(s_val[j + u - j0]) : to_arith(sval[j + u]);
    }
    A y[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) load_row<VS, R>(ycur + (size_t)cj[u] * R, y[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < R; ++t) s[t] = fma(a[u], y[u][t], s[t]);
  }
  for (; j < je; ++j) {
    const int cj = staged ? s_col[j - j0] : __ldg(col + j);
    const A a = staged ? to_arith(s_val[j - j0]) : to_arith(sval[j]);
    A y[R];
    load_row<VS, R>(ycur + (size_t)cj * R, y);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = fma(a, y[t], s[t]);
  }
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] *= A(0.5);
  }
  store_row_rounded<VS, R>(ynext + (size_t)row * R, s);
  const A bn = A(coef[(size_t)(k + 1) * count + pi]);
  A acc[R];
  if (FIRST) {
    A v0[R];
    load_row<VS, R>(ycur + (size_t)row * R, v0);
    const A b0 = A(coef[pi]);
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = b0 * v0[t];
  } else {
    load_acc<R>(acc_io + (size_t)row * R, acc);
  }
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = fma(bn, s[t], acc[t]);
  store_acc<R>(acc_io + (size_t)row * R, acc);
}

// vbuf = Q_j in the filter's storage precision (j from the device step index).
template <class VS>
__global__ void load_block_kernel(const double* __restrict__ Q, const int* __restrict__ jdev, long long nr,
                                  VS* __restrict__ vbuf) {
  const double* src = Q + (size_t)(*jdev) * nr;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (long long)gridDim.x * blockDim.x)
    vbuf[i] = from_arith<VS>((typename Arith<VS>::type)src[i]);
}

__global__ void narrow_df_kernel(const dev::dfloat* __restrict__ in, double* __restrict__ out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = dev::to_double(in[i]);
}

__global__ void widen_kernel(const float* __restrict__ in, double* __restrict__ out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// Partial Q^T W over one chunk (blockIdx.x) for a group of basis blocks (blockIdx.y).
template <int R>
__global__ void __launch_bounds__(kT) seg_dot_kernel(const double* __restrict__ Q, int nb_fixed,
                                                     const int* __restrict__ jdev, long long N,
                                                     const double* __restrict__ W, const int* __restrict__ crow0,
                                                     const int* __restrict__ crow1, const int* __restrict__ cmat,
                                                     const int* __restrict__ active, double* __restrict__ part,
                                                     int nbmax) {
  constexpr int BPW = (8 / R) > 0 ? (8 / R) : 1;
  constexpr int RPI = 32 / R;
  __shared__ double wsm[kSubB * R];
  const int nb = nb_fixed > 0 ? nb_fixed : (*jdev + 1);
  const int ch = blockIdx.x;
  if (!active[cmat[ch]] || (int)blockIdx.y * 8 * BPW >= nb) return;  // uniform over the CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = lane % R, k = lane / R;
  const bool act = k < RPI;
  const long long r0 = crow0[ch], r1 = crow1[ch];
  const int bbase = blockIdx.y * (8 * BPW) + warp * BPW;
  double acc[BPW][R];
#pragma unroll
  for (int bi = 0; bi < BPW; ++bi)
#pragma unroll
    for (int t = 0; t < R; ++t) acc[bi][t] = 0.0;
  for (long long s0 = r0; s0 < r1; s0 += kSubB) {
    const int rows = (int)min((long long)kSubB, r1 - s0);
    for (int e = threadIdx.x; e < rows * R; e += kT) wsm[e] = W[(size_t)s0 * R + e];
    __syncthreads();
    if (act) {
#pragma unroll
      for (int bi = 0; bi < BPW; ++bi) {
        const int b = bbase + bi;
        if (b < nb) {
          const double* qb = Q + (size_t)b * N * R + (size_t)s0 * R;
          for (int i = k; i < rows; i += RPI) {
            const double q = __ldg(qb + (size_t)i * R + a);
#pragma unroll
            for (int t = 0; t < R; ++t) acc[bi][t] = fma(q, wsm[i * R + t], acc[bi][t]);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int bi = 0; bi < BPW; ++bi) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      double v = acc[bi][t];
      for (int s = 1; s < RPI; s <<= 1) {
        const double o = __shfl_down_sync(0xffffffffu, v, s * R);
        if ((k & (2 * s - 1)) == 0 && k + s < RPI) v += o;
      }
      acc[bi][t] = v;
    }
  }
  if (k == 0) {
#pragma unroll
    for (int bi = 0; bi < BPW; ++bi) {
      const int b = bbase + bi;
      if (b < nb) {
        double* p = part + ((size_t)ch * nbmax + b) * R * R + a * R;
#pragma unroll
        for (int t = 0; t < R; ++t) p[t] = acc[bi][t];
      }
    }
  }
}

// C[i][b][a][t] = sum over problem i's chunks of part[chunk][b][a][t].
__global__ void seg_reduce_kernel(int count, int r, int nb_fixed, const int* __restrict__ jdev, int nbmax,
                                  const int* __restrict__ cbeg, const int* __restrict__ active,
                                  const double* __restrict__ part, double* __restrict__ C) {
  const int nb = nb_fixed > 0 ? nb_fixed : (*jdev + 1);
  const long long per = (long long)nb * r * r;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < (long long)count * per;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o / per);
    if (!active[i]) continue;
    const long long w = o - (long long)i * per;  // index within [nb][r][r]
    double s = 0.0;
    for (int c = cbeg[i]; c < cbeg[i + 1]; ++c) s += part[(size_t)c * nbmax * r * r + w];
    C[(size_t)i * nbmax * r * r + w] = s;
  }
}

// Out[row, t] = beta Out + alpha sum_{b<nb, a<r} Q_b[row, a] C_i[(b r + a) S + t], i = problem of row.
template <int S>
__global__ void __launch_bounds__(kT) seg_update_kernel(const double* Q, int nb_fixed, const int* __restrict__ jdev,
                                                        long long N, int r, const double* __restrict__ C,
                                                        long long cstride, double alpha, double beta, double* Out,
                                                        int ldo, const int* __restrict__ off, int count,
                                                        const int* __restrict__ active) {
  extern __shared__ int s_off2[];
  for (int i = threadIdx.x; i <= count; i += kT) s_off2[i] = off[i];
  __syncthreads();
  const long long row = (long long)blockIdx.x * kT + threadIdx.x;
  if (row >= N) return;
  const int pi = problem_of(s_off2, count, (int)row);
  if (!active[pi]) return;
  const int nb = nb_fixed > 0 ? nb_fixed : (*jdev + 1);
  const double* Ci = C + (size_t)pi * cstride;
  double acc[S];
#pragma unroll
  for (int t = 0; t < S; ++t) acc[t] = 0.0;
  for (int b = 0; b < nb; ++b) {
    const double* qrow = Q + (size_t)b * N * r + (size_t)row * r;
    for (int a = 0; a < r; ++a) {
      const double q = qrow[a];
      const double* cr = Ci + (size_t)(b * r + a) * S;
#pragma unroll
      for (int t = 0; t < S; ++t) acc[t] = fma(q, __ldg(cr + t), acc[t]);
    }
  }
  double* o = Out + (size_t)row * ldo;
  if (beta == 0.0) {
#pragma unroll
    for (int t = 0; t < S; ++t) o[t] = alpha * acc[t];
  } else {
#pragma unroll
    for (int t = 0; t < S; ++t) o[t] = fma(alpha, acc[t], beta * o[t]);
  }
}

// Block QR factor of every active problem from its Gram matrix G_i (r x r):
// Cholesky (shifted on pass 0, as in shifted CholeskyQR3), R^{-1} for the
// scaling update, and S_i <- R S_i (S_i = R on pass 0). One thread per problem.
__global__ void seg_chol_kernel(int count, int r, int nbmax, const int* __restrict__ active,
                                const int* __restrict__ off, const double* __restrict__ G, double* __restrict__ Rinv,
                                double* __restrict__ Sacc, int pass, int* __restrict__ fail_flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count || !active[i]) return;
  const double* g = G + (size_t)i * nbmax * r * r;  // block 0 of problem i's C layout
  double R[16 * 16], Ri[16 * 16];
  double gmax = 0.0;
  for (int d = 0; d < r; ++d) gmax = fmax(gmax, g[d * r + d]);
  const double nrows = (double)(off[i + 1] - off[i]);
  const double shift = pass == 0 ? 11.0 * (nrows * r + (double)r * (r + 1)) * 1.1102230246251565e-16 * fmax(gmax * r, 1e-300) : 0.0;
  for (int a = 0; a < r * r; ++a) R[a] = 0.0;
  for (int a = 0; a < r; ++a) {
    double d = g[a * r + a] + shift;
    for (int q = 0; q < a; ++q) d -= R[q * r + a] * R[q * r + a];
    if (!(d > 0.0)) {
      atomicOr(fail_flag, 1);
      d = fmax(1e-300, fabs(d));
    }
    const double rd = sqrt(d);
    R[a * r + a] = rd;
    for (int b = a + 1; b < r; ++b) {
      double v = g[a * r + b];
      for (int q = 0; q < a; ++q) v -= R[q * r + a] * R[q * r + b];
      R[a * r + b] = v / rd;
    }
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
  double* ri = Rinv + (size_t)i * r * r;
  for (int a = 0; a < r * r; ++a) ri[a] = Ri[a];
  double* sa = Sacc + (size_t)i * r * r;
  if (pass == 0) {
    for (int a = 0; a < r * r; ++a) sa[a] = R[a];
  } else {
    double T[16 * 16];
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) {
        double v = 0.0;
        for (int q = 0; q < r; ++q) v += R[a * r + q] * sa[q * r + b];
        T[a * r + b] = v;
      }
    for (int a = 0; a < r * r; ++a) sa[a] = T[a];
  }
}

// D history: Dh[i][j] = C1[i][j] + C2[i][j] (the total projection on Q_j).
__global__ void d_history_kernel(int count, int r, int nbmax, const int* __restrict__ jdev,
                                 const int* __restrict__ active, const double* __restrict__ C1,
                                 const double* __restrict__ C2, double* __restrict__ Dh) {
  const int j = *jdev;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < count * r * r; o += gridDim.x * blockDim.x) {
    const int i = o / (r * r), w = o - i * r * r;
    if (!active[i]) continue;
    const size_t at = ((size_t)i * nbmax + j) * r * r + w;
    Dh[at] = C1[at] + C2[at];
  }
}

// S history and the new basis block: Sh[i][j] = S_i; Q_{j+1} = W; then j += 1.
__global__ void s_history_kernel(int count, int r, int nbmax, const int* __restrict__ jdev,
                                 const int* __restrict__ active, const double* __restrict__ Sacc,
                                 double* __restrict__ Sh) {
  const int j = *jdev;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < count * r * r; o += gridDim.x * blockDim.x) {
    const int i = o / (r * r), w = o - i * r * r;
    if (!active[i]) continue;
    Sh[((size_t)i * nbmax + j) * r * r + w] = Sacc[o];
  }
}

__global__ void store_block_kernel(const double* __restrict__ W, double* __restrict__ Q, const int* __restrict__ jdev,
                                   int offset, int nbmax, long long nr) {
  const int b = *jdev + offset;
  if (b < 0 || b >= nbmax) return;
  double* dst = Q + (size_t)b * nr;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (long long)gridDim.x * blockDim.x)
    dst[i] = W[i];
}

__global__ void advance_kernel(int* jdev) { *jdev += 1; }

// out[j] = (2/e_i)(val[j] - c_i [j diagonal]) for the problem i of the row.
template <class S>
__global__ void seg_scale_kernel(long long N, const int* __restrict__ rowptr, const int* __restrict__ diag_pos,
                                 const double* __restrict__ val, const int* __restrict__ off, int count,
                                 const double* __restrict__ cc, const double* __restrict__ ee, S* __restrict__ out) {
  extern __shared__ int s_off3[];
  for (int i = threadIdx.x; i <= count; i += blockDim.x) s_off3[i] = off[i];
  __syncthreads();
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < N; row += (long long)gridDim.x * blockDim.x) {
    const int pi = problem_of(s_off3, count, (int)row);
    const double s = 2.0 / ee[pi], c = cc[pi];
    const int d = diag_pos[row];
    for (int j = rowptr[row], je = rowptr[row + 1]; j < je; ++j) {
      const double v = s * (val[j] - (j == d ? c : 0.0));
      if constexpr (std::is_same<S, double>::value) out[j] = v;
      else if constexpr (std::is_same<S, float>::value) out[j] = (float)v;
      else if constexpr (std::is_same<S, dev::dfloat>::value) out[j] = dev::dfloat(v);
      else out[j] = __double2bfloat16(v);
    }
  }
}

// Y = A X on the concatenated matrix (FP64 values), X, Y n x s with stride ld.
__global__ void seg_spmm_kernel(long long N, int s, int ld, const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ X, double* __restrict__ Y) {
  const int rpw = 32 / s;
  const int lane = threadIdx.x & 31;
  const int sub = lane / s, c = lane - sub * s;
  const long long row = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * rpw + sub;
  if (sub >= rpw || row >= N) return;
  double acc = 0.0;
  for (int j = rowptr[row], je = rowptr[row + 1]; j < je; ++j) acc = fma(val[j], X[(size_t)col[j] * ld + c], acc);
  Y[(size_t)row * ld + c] = acc;
}

// Per-chunk column sums of X*Y (mode 0) or (Y - lam_i X)^2 (mode 1), 16 columns.
__global__ void seg_colsum_kernel(const double* __restrict__ X, const double* __restrict__ Y,
                                  const double* __restrict__ lam, int mode, const int* __restrict__ crow0,
                                  const int* __restrict__ crow1, const int* __restrict__ cmat,
                                  const int* __restrict__ walking, double* __restrict__ part) {
  __shared__ double red[kT];
  const int ch = blockIdx.x;
  const int pi = cmat[ch];
  if (!walking[pi]) return;
  const int t = threadIdx.x & 15, sub = threadIdx.x >> 4;  // 16 rows per pass
  const double l = mode == 1 ? lam[pi * 16 + t] : 0.0;
  double acc = 0.0;
  for (long long row = crow0[ch] + sub; row < crow1[ch]; row += kT / 16) {
    const double x = X[(size_t)row * 16 + t], y = Y[(size_t)row * 16 + t];
    if (mode == 0) acc = fma(x, y, acc);
    else {
      const double d = y - l * x;
      acc = fma(d, d, acc);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < 16) {
    double v = 0.0;
    for (int q = 0; q < kT / 16; ++q) v += red[q * 16 + threadIdx.x];
    part[(size_t)ch * 16 + threadIdx.x] = v;
  }
}

__global__ void seg_colsum_reduce_kernel(int count, const int* __restrict__ cbeg, const int* __restrict__ walking,
                                         const double* __restrict__ part, double* __restrict__ out) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < count * 16; o += gridDim.x * blockDim.x) {
    const int i = o / 16, t = o - i * 16;
    if (!walking[i]) continue;
    double s = 0.0;
    for (int c = cbeg[i]; c < cbeg[i + 1]; ++c) s += part[(size_t)c * 16 + t];
    out[o] = s;
  }
}

__global__ void offset_copy_kernel(const int* __restrict__ src, int* __restrict__ dst, long long count, int add) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] < 0 ? src[i] : src[i] + add;
}

__global__ void seg_random_kernel(double* __restrict__ X, long long count, uint64_t seed) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x) {
    uint64_t z = seed ^ (0x9e3779b97f4a7c15ull * (uint64_t)(2 * k + 1));
    auto mix = [](uint64_t v) {
      v += 0x9e3779b97f4a7c15ull;
      v = (v ^ (v >> 30)) * 0xbf58476d1ce4e5b9ull;
      v = (v ^ (v >> 27)) * 0x94d049bb133111ebull;
      return v ^ (v >> 31);
    };
    const double u1 = ((double)(mix(z) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(mix(z + 1) >> 11) * (1.0 / 9007199254740992.0);
    X[k] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

inline unsigned gsb(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

#define FLZ_DISPATCH_R(r, FN, ...)                                 \
  switch (r) {                                                     \
    case 1: FN<1>(__VA_ARGS__); break;                             \
    case 2: FN<2>(__VA_ARGS__); break;                             \
    case 4: FN<4>(__VA_ARGS__); break;                             \
    case 8: FN<8>(__VA_ARGS__); break;                             \
    case 16: FN<16>(__VA_ARGS__); break;                           \
    default: fail(FLZ_ERR_INVALID_ARG, "batch block size %d not in {1,2,4,8,16}", r); \
  }

// All device state of one lockstep run (bounds phase or main phase).
struct BatchEngine {
  flz_batch* B;
  int r, nbmax, count;
  long long N;
  cudaStream_t st;
  int precision;
  DevBuf<double> Q, W, C1, C2, G, Rinv, Sacc, Dh, Sh, part, coef, cc, ee;
  DevBuf<float> acc32, v32, ya32, yb32;
  DevBuf<__nv_bfloat16> v16, ya16, yb16;
  DevBuf<double> ya64, yb64, sval64;
  DevBuf<float> sval32;
  DevBuf<__nv_bfloat16> sval16;
  DevBuf<dev::dfloat> svaldf, vdf, yadf, ybdf, accdf;  // double-FP32 filter
  DevBuf<int> jdev, active, mdeg, fail;
  int mmax = 0;
  bool pdl = true;  // degree steps as programmatic dependent launches
  bool persistent = false;  // fixed-point filter: every degree in one cooperative launch
  int n_chunks = 0;

  void setup(flz_batch* b, int r_, int nbmax_, int prec, cudaStream_t s) {
    B = b;
    r = r_;
    nbmax = nbmax_;
    count = b->count;
    N = b->N;
    st = s;
    precision = prec;
    n_chunks = (int)b->c_mat.size();
    const size_t nr = (size_t)N * r;
    Q.reserve((size_t)nbmax * nr);
    W.reserve(nr);
    const size_t cs = (size_t)count * nbmax * r * r;
    C1.reserve(cs);
    C2.reserve(cs);
    G.reserve(cs);
    Dh.reserve(cs);
    Sh.reserve(cs);
    Rinv.reserve((size_t)count * r * r);
    Sacc.reserve((size_t)count * r * r);
    part.reserve((size_t)n_chunks * nbmax * r * r);
    jdev.reserve(1);
    active.reserve(count);
    mdeg.reserve(count);
    fail.reserve(1);
    cc.reserve(count);
    ee.reserve(count);
    if (prec == FLZ_PREC_FP64) {
      v64.reserve(nr);
      ya64.reserve(nr);
      yb64.reserve(nr);
      sval64.reserve((size_t)b->nnz);
    } else if (prec == FLZ_PREC_FP32) {
      acc32.reserve(nr);
      v32.reserve(nr);
      ya32.reserve(nr);
      yb32.reserve(nr);
      sval32.reserve((size_t)b->nnz);
    } else if (prec == FLZ_PREC_DF64) {
      accdf.reserve(nr);
      vdf.reserve(nr);
      yadf.reserve(nr);
      ybdf.reserve(nr);
      svaldf.reserve((size_t)b->nnz);
    } else {
      acc32.reserve(nr);
      v16.reserve(nr);
      ya16.reserve(nr);
      yb16.reserve(nr);
      sval16.reserve((size_t)b->nnz);
    }
  }

  void set_filter(const std::vector<double>& c, const std::vector<double>& e, const std::vector<std::vector<double>>& coeffs) {
    mmax = 0;
    for (auto& v : coeffs) mmax = std::max(mmax, (int)v.size() - 1);
    std::vector<double> table((size_t)(mmax + 1) * count, 0.0);
    std::vector<int> m(count);
    for (int i = 0; i < count; ++i) {
      m[i] = (int)coeffs[i].size() - 1;
      for (int k = 0; k <= m[i]; ++k) table[(size_t)k * count + i] = coeffs[i][k];
    }
    coef.reserve(table.size());
    FLZ_CUDA(cudaMemcpyAsync(coef.p, table.data(), sizeof(double) * table.size(), cudaMemcpyHostToDevice, st));
    FLZ_CUDA(cudaMemcpyAsync(mdeg.p, m.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
    FLZ_CUDA(cudaMemcpyAsync(cc.p, c.data(), sizeof(double) * count, cudaMemcpyHostToDevice, st));
    FLZ_CUDA(cudaMemcpyAsync(ee.p, e.data(), sizeof(double) * count, cudaMemcpyHostToDevice, st));
    if (precision == FLZ_PREC_FX64) {
      // the fixed-point filter where its format holds every problem, else FP64
      if (fx_batch_prepare(B->fxb, N, B->nnz, B->rowptr.p, B->col.p, B->val.p, B->diag_pos.p, B->max_row_nnz,
                           B->d_off.p, B->off, count, cc.p, ee.p, r, st) &&
          fx_batch_coefficients(B->fxb, coeffs, st))
        return;
      precision = FLZ_PREC_FP64;
      const size_t nr = (size_t)N * r;
      v64.reserve(nr);
      ya64.reserve(nr);
      yb64.reserve(nr);
      sval64.reserve((size_t)B->nnz);
    }
    const size_t sm = sizeof(int) * (count + 1);
    if (precision == FLZ_PREC_FP64)
      seg_scale_kernel<double><<<gsb(N), 256, sm, st>>>(N, B->rowptr.p, B->diag_pos.p, B->val.p, B->d_off.p, count, cc.p, ee.p, sval64.p);
    else if (precision == FLZ_PREC_FP32)
      seg_scale_kernel<float><<<gsb(N), 256, sm, st>>>(N, B->rowptr.p, B->diag_pos.p, B->val.p, B->d_off.p, count, cc.p, ee.p, sval32.p);
    else if (precision == FLZ_PREC_DF64)
      seg_scale_kernel<dev::dfloat><<<gsb(N), 256, sm, st>>>(N, B->rowptr.p, B->diag_pos.p, B->val.p, B->d_off.p, count, cc.p, ee.p, svaldf.p);
    else
      seg_scale_kernel<__nv_bfloat16><<<gsb(N), 256, sm, st>>>(N, B->rowptr.p, B->diag_pos.p, B->val.p, B->d_off.p, count, cc.p, ee.p, sval16.p);
    FLZ_LAUNCH_CHECK();
  }

  void set_active(const std::vector<int>& act) {
    FLZ_CUDA(cudaMemcpyAsync(active.p, act.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  }

  template <int R>
  void dot(const double* Qp, int nb_fixed, const double* Wp, double* Cout) {
    const int bpc = 8 * std::max(1, 8 / R);
    const int groups = (nb_fixed > 0 ? nb_fixed + bpc - 1 : nbmax + bpc - 1) / bpc;
    seg_dot_kernel<R><<<dim3(n_chunks, groups), kT, 0, st>>>(Qp, nb_fixed, jdev.p, N, Wp, B->d_c_row0.p, B->d_c_row1.p,
                                                              B->d_c_mat.p, active.p, part.p, nbmax);
    FLZ_LAUNCH_CHECK();
    const long long outs = (long long)count * (nb_fixed > 0 ? nb_fixed : nbmax) * R * R;
    seg_reduce_kernel<<<gsb(outs), 256, 0, st>>>(count, R, nb_fixed, jdev.p, nbmax, B->d_c_beg.p, active.p, part.p, Cout);
    FLZ_LAUNCH_CHECK();
  }

  template <int S>
  void update(const double* Qp, int nb_fixed, int rr, const double* C, long long cstride, double alpha, double beta,
              double* Out, int ldo, const int* act) {
    const size_t sm = sizeof(int) * (count + 1);
    seg_update_kernel<S><<<(unsigned)((N + kT - 1) / kT), kT, sm, st>>>(Qp, nb_fixed, jdev.p, N, rr, C, cstride, alpha, beta,
                                                                      Out, ldo, B->d_off.p, count, act);
    FLZ_LAUNCH_CHECK();
  }

  template <int R, class MS, class VS, class AccS>
  void filter_steps(const MS* sv, VS* v, VS* ya, VS* yb, AccS* acc) {
    // staging capacity chosen so the dynamic shared memory stays within 48 KB
    const long long room = 48 * 1024 - 64 - (long long)sizeof(int) * (count + 1);
    const int cap = (int)std::max<long long>(0, std::min<long long>(B->max_cta_nnz, room / (long long)(sizeof(MS) + sizeof(int))));
    const size_t sm = (size_t)cap * (sizeof(MS) + sizeof(int)) + sizeof(int) * (count + 1) + 16;
    const unsigned grid = (unsigned)((N + kRowsB - 1) / kRowsB);
    const int* rp = B->rowptr.p;
    const int* cl = B->col.p;
    seg_cheb_kernel<R, MS, VS, AccS, true><<<grid, kRowsB, sm, st>>>((int)N, cap, rp, cl, sv, B->d_off.p, count, coef.p, 0,
                                                                     mdeg.p, active.p, v, nullptr, ya, acc);
    FLZ_LAUNCH_CHECK();
    const VS* prev = v;
    const VS* cur = ya;
    for (int k = 1; k < mmax; ++k) {
      VS* next = (k == 1) ? yb : const_cast<VS*>(prev);
      // degrees after the first overlap their staging with the previous
      // degree's tail (programmatic dependent launch, captured into the graph)
      if (pdl)
        launch_dependent(seg_cheb_kernel<R, MS, VS, AccS, false>, grid, kRowsB, sm, st, (int)N, cap, rp, cl, sv,
                         B->d_off.p, count, coef.p, k, mdeg.p, active.p, cur, prev, next, acc);
      else
        seg_cheb_kernel<R, MS, VS, AccS, false><<<grid, kRowsB, sm, st>>>((int)N, cap, rp, cl, sv, B->d_off.p, count,
                                                                          coef.p, k, mdeg.p, active.p, cur, prev, next, acc);
      FLZ_LAUNCH_CHECK();
      prev = cur;
      cur = next;
    }
  }

  // W = p_i(Ahat_i) Q_j for every active problem.
  template <int R>
  void apply_filter() {
    const long long nr = N * R;
    if (precision == FLZ_PREC_FX64) {
      fx_batch_filter(B->fxb, R, Q.p, jdev.p, B->d_off.p, mdeg.p, active.p, W.p, pdl, persistent, st);
    } else if (precision == FLZ_PREC_FP64) {
      // V = Q_j in a fixed buffer (the graph is replayed with a moving j); the sum is W
      load_block_kernel<double><<<gsb(nr), 256, 0, st>>>(Q.p, jdev.p, nr, v64.p);
      FLZ_LAUNCH_CHECK();
      filter_steps<R, double, double, double>(sval64.p, v64.p, ya64.p, yb64.p, W.p);
    } else if (precision == FLZ_PREC_FP32) {
      load_block_kernel<float><<<gsb(nr), 256, 0, st>>>(Q.p, jdev.p, nr, v32.p);
      FLZ_LAUNCH_CHECK();
      filter_steps<R, float, float, float>(sval32.p, v32.p, ya32.p, yb32.p, acc32.p);
      widen_kernel<<<gsb(nr), 256, 0, st>>>(acc32.p, W.p, nr);
      FLZ_LAUNCH_CHECK();
    } else if (precision == FLZ_PREC_DF64) {
      load_block_kernel<dev::dfloat><<<gsb(nr), 256, 0, st>>>(Q.p, jdev.p, nr, vdf.p);
      FLZ_LAUNCH_CHECK();
      filter_steps<R, dev::dfloat, dev::dfloat, dev::dfloat>(svaldf.p, vdf.p, yadf.p, ybdf.p, accdf.p);
      narrow_df_kernel<<<gsb(nr), 256, 0, st>>>(accdf.p, W.p, nr);
      FLZ_LAUNCH_CHECK();
    } else {
      load_block_kernel<__nv_bfloat16><<<gsb(nr), 256, 0, st>>>(Q.p, jdev.p, nr, v16.p);
      FLZ_LAUNCH_CHECK();
      filter_steps<R, __nv_bfloat16, __nv_bfloat16, float>(sval16.p, v16.p, ya16.p, yb16.p, acc32.p);
      widen_kernel<<<gsb(nr), 256, 0, st>>>(acc32.p, W.p, nr);
      FLZ_LAUNCH_CHECK();
    }
  }

  DevBuf<double> v64;

  // Tensor-core reorthogonalization: each problem keeps its own digit copy of
  // its basis (grown as the basis grows) and the projections and updates run
  // per problem, host-driven between the two captured halves of a step.
  // The problems' kernels are small; they run on kSide side streams (problem
  // i on stream i % kSide), forked from and joined back into the main stream.
  static constexpr int kSide = 8;
  bool tc = false;
  std::vector<std::unique_ptr<TcBasis>> tcb;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};

  void setup_tc(int64_t kcap0) {
    tcb.clear();
    for (int i = 0; i < count; ++i) {
      tcb.emplace_back(new TcBasis());
      tcb[i]->reserve(B->off[i + 1] - B->off[i], std::min<int64_t>(kcap0, (int64_t)nbmax * r));
    }
    FLZ_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    for (int q = 0; q < kSide; ++q) {
      FLZ_CUDA(cudaStreamCreateWithFlags(&side[q], cudaStreamNonBlocking));
      FLZ_CUDA(cudaEventCreateWithFlags(&join_ev[q], cudaEventDisableTiming));
    }
    tc = true;
  }
  ~BatchEngine() {
    for (int q = 0; q < kSide; ++q) {
      if (side[q]) cudaStreamSynchronize(side[q]), cudaStreamDestroy(side[q]);
      if (join_ev[q]) cudaEventDestroy(join_ev[q]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
  }
  // runs f(i, stream) for the active problems on the side streams, ordered
  // after everything on the main stream and before anything issued to it later
  template <class F>
  void on_side_streams(const std::vector<int>& act, F f) {
    FLZ_CUDA(cudaEventRecord(fork_ev, st));
    for (int q = 0; q < kSide; ++q) FLZ_CUDA(cudaStreamWaitEvent(side[q], fork_ev, 0));
    for (int i = 0; i < count; ++i)
      if (act[i]) f(i, side[i % kSide]);
    for (int q = 0; q < kSide; ++q) {
      FLZ_CUDA(cudaEventRecord(join_ev[q], side[q]));
      FLZ_CUDA(cudaStreamWaitEvent(st, join_ev[q], 0));
    }
  }
  // CGS2 of every active problem's W against its K basis columns, writing the
  // two projections where the history kernels read them.
  void tc_orth(int K, const std::vector<int>& act) {
    const size_t cs = (size_t)nbmax * r * r;
    on_side_streams(act, [&](int i, cudaStream_t s) {
      tcb[i]->cgs2(K, W.p + (size_t)B->off[i] * r, r, C1.p + i * cs, C2.p + i * cs, s);
    });
  }
  // Digits of the newest block (index col0 / r, just stored) of every active problem.
  void tc_append(int col0, const std::vector<int>& act) {
    const double* blk = Q.p + (size_t)(col0 / r) * N * r;
    on_side_streams(act, [&](int i, cudaStream_t s) {
      tcb[i]->grow(col0 + r, s);
      tcb[i]->append(const_cast<double*>(blk) + (size_t)B->off[i] * r, r, col0, s);
    });
  }
  // raises FLZ_ERR_TIMEOUT if a tensor-core wait expired (after a stream sync)
  void tc_check() {
    for (auto& t : tcb) t->check_status();
  }

  // One block Lanczos step for every active problem (graph-capturable).
  template <int R>
  void step() {
    apply_filter<R>();
    step_after_filter<R>();
  }

  // CUDA-core CGS2 and the rest of the step after the filter
  template <int R>
  void step_after_filter() {
    // CGS2 against Q_0..Q_j (nb from the device step index)
    dot<R>(Q.p, 0, W.p, C1.p);
    update<R>(Q.p, 0, R, C1.p, (long long)nbmax * R * R, -1.0, 1.0, W.p, R, active.p);
    dot<R>(Q.p, 0, W.p, C2.p);
    update<R>(Q.p, 0, R, C2.p, (long long)nbmax * R * R, -1.0, 1.0, W.p, R, active.p);
    step_tail<R>();
  }

  // The part of a step after the reorthogonalization: projection history,
  // block QR, S history, the new basis block, the step index.
  template <int R>
  void step_tail() {
    d_history_kernel<<<gsb((long long)count * R * R), 256, 0, st>>>(count, R, nbmax, jdev.p, active.p, C1.p, C2.p, Dh.p);
    FLZ_LAUNCH_CHECK();
    qr<R>();
    s_history_kernel<<<gsb((long long)count * R * R), 256, 0, st>>>(count, R, nbmax, jdev.p, active.p, Sacc.p, Sh.p);
    FLZ_LAUNCH_CHECK();
    store_block_kernel<<<gsb(N * R), 256, 0, st>>>(W.p, Q.p, jdev.p, 1, nbmax, N * R);
    FLZ_LAUNCH_CHECK();
    advance_kernel<<<1, 1, 0, st>>>(jdev.p);
    FLZ_LAUNCH_CHECK();
  }

  // Shifted CholeskyQR3 of W in place; S_i accumulated in Sacc.
  template <int R>
  void qr() {
    for (int pass = 0; pass < 3; ++pass) {
      dot<R>(W.p, 1, W.p, G.p);
      seg_chol_kernel<<<(count + 127) / 128, 128, 0, st>>>(count, R, nbmax, active.p, B->d_off.p, G.p, Rinv.p, Sacc.p,
                                                           pass, fail.p);
      FLZ_LAUNCH_CHECK();
      update<R>(W.p, 1, R, Rinv.p, (long long)R * R, 1.0, 0.0, W.p, R, active.p);
    }
  }

  template <int R>
  void start_block(uint64_t seed) {
    seg_random_kernel<<<gsb(N * R), 256, 0, st>>>(W.p, N * R, seed);
    FLZ_LAUNCH_CHECK();
    qr<R>();
    int m1 = -1;
    FLZ_CUDA(cudaMemcpyAsync(jdev.p, &m1, sizeof(int), cudaMemcpyHostToDevice, st));
    store_block_kernel<<<gsb(N * R), 256, 0, st>>>(W.p, Q.p, jdev.p, 1, nbmax, N * R);
    FLZ_LAUNCH_CHECK();
    advance_kernel<<<1, 1, 0, st>>>(jdev.p);
    FLZ_LAUNCH_CHECK();
    FLZ_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), st));
  }
};

struct WalkState {
  int inside = 0, outside = 0;
  bool all_small = true, done = false;
  int walked = 0;
  std::vector<double> vals, res;
  std::vector<int> order;
  std::vector<double> theta, T;
  int K = 0;
  std::vector<double> walkY;  // eigenvectors of T formed so far in this check
  std::vector<int> walkIdx;
};

}  // namespace

namespace {

void build_chunks(flz_batch* b) {
  const int target = (int)std::max<int64_t>(kSubB, (b->N + 1023) / 1024);
  const int rows = (target + kSubB - 1) / kSubB * kSubB;
  b->c_row0.clear();
  b->c_row1.clear();
  b->c_mat.clear();
  b->c_beg.assign(b->count + 1, 0);
  for (int i = 0; i < b->count; ++i) {
    b->c_beg[i] = (int)b->c_mat.size();
    for (int r0 = b->off[i]; r0 < b->off[i + 1]; r0 += rows) {
      b->c_row0.push_back(r0);
      b->c_row1.push_back(std::min(b->off[i + 1], r0 + rows));
      b->c_mat.push_back(i);
    }
  }
  b->c_beg[b->count] = (int)b->c_mat.size();
  auto up = [](DevBuf<int>& d, const std::vector<int>& h) {
    d.reserve(std::max<size_t>(h.size(), 1));
    FLZ_CUDA(cudaMemcpy(d.p, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice));
  };
  up(b->d_c_row0, b->c_row0);
  up(b->d_c_row1, b->c_row1);
  up(b->d_c_mat, b->c_mat);
  up(b->d_c_beg, b->c_beg);
}

// Host view of problem i's projected matrix after k steps.
std::vector<double> assemble_T(const std::vector<double>& Dh, const std::vector<double>& Sh, int i, int k, int r,
                               int nbmax) {
  const int K = k * r;
  std::vector<double> T((size_t)K * K, 0.0);
  for (int b = 0; b < k; ++b) {
    const double* D = &Dh[((size_t)i * nbmax + b) * r * r];
    for (int a = 0; a < r; ++a)
      for (int c = 0; c < r; ++c) T[(size_t)(b * r + a) * K + b * r + c] = 0.5 * (D[a * r + c] + D[c * r + a]);
    if (b + 1 < k) {
      const double* S = &Sh[((size_t)i * nbmax + b) * r * r];
      for (int a = 0; a < r; ++a)
        for (int c = 0; c < r; ++c) {
          T[(size_t)((b + 1) * r + a) * K + b * r + c] = S[a * r + c];
          T[(size_t)(b * r + c) * K + (b + 1) * r + a] = S[a * r + c];
        }
    }
  }
  return T;
}

template <class F>
void parallel_for(int n, F f) {
  const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int i = t; i < n; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

template <int R>
void run_lockstep(BatchEngine& E, int steps) {
  for (int s = 0; s < steps; ++s) E.step<R>();
}

// Captures one block step of E into an executable graph. Nothing in a step
// allocates or synchronizes; if anything fails the capture is ended before
// the error propagates, so the stream is usable again.
template <class F>
cudaGraphExec_t capture_once(BatchEngine& E, F part) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  FLZ_CUDA(cudaStreamBeginCapture(E.st, cudaStreamCaptureModeThreadLocal));
  try {
    part();
  } catch (...) {
    cudaGraph_t partial = nullptr;
    cudaStreamEndCapture(E.st, &partial);
    if (partial) cudaGraphDestroy(partial);
    cudaGetLastError();
    throw;
  }
  FLZ_CUDA(cudaStreamEndCapture(E.st, &g));
  const cudaError_t err = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  FLZ_CUDA(err);
  return ge;
}

// Captures part of a block step; if the programmatic dependent launches
// cannot be captured, captures again with plain launches.
template <class F>
cudaGraphExec_t capture_part(BatchEngine& E, F part) {
  try {
    return capture_once(E, part);
  } catch (const Failure&) {
    if (!E.pdl) throw;
    cudaGetLastError();
    E.pdl = false;
    return capture_once(E, part);
  }
}

// The mixed-precision batch: each converged problem's pairs (FP32 / BF16
// filter quality) are refined to params.tol by filtered subspace iteration
// with the fixed-point filter on its own matrix and Rayleigh-Ritz on A (the
// single solve's refinement). The block is the found eigenvectors plus guard
// and extra random columns (the extras are filtered with the problem's
// filter at half degree in the first sweep). The problems are small and a
// refinement is a few hundred small launches with host synchronizations, so
// up to eight host threads run them, each on its own stream with its own
// workspace sized for the largest problem beforehand (nothing is allocated
// or freed per problem: cudaFree would synchronize the whole device).
struct RefineSlot {
  cudaStream_t st = nullptr;
  RefineWorkspace ws;
  DevBuf<double> X, dv, prt;
  std::vector<double> nrm2;
  ~RefineSlot() {
    if (st) cudaStreamSynchronize(st), cudaStreamDestroy(st);
  }
};

int refine_block_width(int64_t f, int guard) {
  const int kp = (int)(f + guard + std::max<int64_t>(16, f / 3));
  return (kp + 15) / 16 * 16;
}

void refine_one(flz_batch* B, int i, const std::vector<double>& coeffs, int guard, RefineSlot& slot) {
  const flz_params& p = B->p;
  cudaStream_t st = slot.st;
  flz_stats& s = B->stats[i];
  const int64_t f = s.count;
  const int64_t n_i = B->off[i + 1] - B->off[i];
  const int kp = refine_block_width(f, guard);
  double* Xr = slot.X.p;
  random_normal(Xr, n_i * kp, p.seed ^ (0x51ull + (uint64_t)i), 0, st);
  columns_to_blocks(B->evecs[i]->p, n_i, n_i, (int)f, Xr, st);
  const int m = s.degree;
  std::vector<double> half;
  if (m >= 8) {
    half.resize(m / 2 + 1);
    filter_coeffs_for(p, s.alpha_mapped, s.beta_mapped, m / 2, half.data());
  }
  RefineArgs ra{B->alpha[i], B->beta[i], s.lmin, s.lmax, p.tol, p.precision == FLZ_PREC_FP32 ? 16 : 24,
                std::max(m, 64), coeffs, half, (int)f};
  ra.flat_first = true;
  const RefineResult rr = refine(B->mats[i], ra, Xr, kp, st, &slot.ws);
  s.refine_sweeps = rr.sweeps;
  s.refine_degree = rr.degrees.empty() ? 0 : *std::max_element(rr.degrees.begin(), rr.degrees.end());
  s.ms_refine = rr.ms;
  s.sweep_matvecs = rr.matvecs;
  // the refined pairs, ascending, as unit columns
  const int64_t g = (int64_t)rr.vals.size();
  std::vector<int> perm(g);
  for (int q = 0; q < g; ++q) perm[q] = q;
  std::sort(perm.begin(), perm.end(), [&](int a, int b) { return rr.vals[a] < rr.vals[b]; });
  slot.nrm2.assign(kp, 1.0);
  for (int b = 0; b < kp / 16; ++b) {
    const double* Xb = Xr + (size_t)b * n_i * 16;
    column_sums(Xb, Xb, nullptr, n_i, 16, 16, 0, slot.dv.p, slot.prt.p, st);
    FLZ_CUDA(cudaMemcpyAsync(slot.nrm2.data() + 16 * b, slot.dv.p, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
  auto& buf = *B->evecs[i];
  if (buf.count < (size_t)std::max<int64_t>(g, 1) * n_i) buf.reserve((size_t)std::max<int64_t>(g, 1) * n_i);
  B->evals[i].resize(g);
  B->resid[i].resize(g);
  double maxres = 0.0;
  for (int64_t q = 0; q < g; ++q) {
    const int col = rr.index[perm[q]];
    rows_to_columns(Xr + (size_t)(col / 16) * n_i * 16 + (col % 16), n_i, 1, 16, buf.p + (size_t)q * n_i, n_i, st,
                    1.0 / std::sqrt(std::max(slot.nrm2[col], 1e-300)));
    B->evals[i][q] = rr.vals[perm[q]];
    B->resid[i][q] = rr.res[perm[q]];
    maxres = std::max(maxres, rr.res[perm[q]]);
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
  s.count = g;
  s.max_residual = maxres;
  s.converged = rr.converged ? 1 : 0;
}

void refine_problems(flz_batch* B, const std::vector<std::vector<double>>& coeffs, const std::vector<int>& converged,
                     int guard) {
  // the problems to refine, largest first (each thread's first is its largest)
  std::vector<int> todo;
  int64_t n_max = 0;
  int kp_max = 16;
  for (int i = 0; i < B->count; ++i) {
    const int64_t f = B->stats[i].count;
    const int64_t n_i = B->off[i + 1] - B->off[i];
    if (!converged[i] || f == 0) continue;
    const int kp = refine_block_width(f, guard);
    if ((int64_t)kp * 4 > n_i) continue;  // too small a problem for a subspace block: its phase result stands
    todo.push_back(i);
    n_max = std::max(n_max, n_i);
    kp_max = std::max(kp_max, kp);
  }
  if (todo.empty()) return;
  std::sort(todo.begin(), todo.end(), [&](int a, int b) { return B->off[a + 1] - B->off[a] > B->off[b + 1] - B->off[b]; });
  const int threads = (int)std::min<size_t>(8, todo.size());
  std::vector<std::unique_ptr<RefineSlot>> slots;
  for (int t = 0; t < threads; ++t) {
    slots.emplace_back(new RefineSlot());
    RefineSlot& sl = *slots.back();
    FLZ_CUDA(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
    sl.X.reserve((size_t)n_max * kp_max);
    sl.dv.reserve(16);
    sl.prt.reserve(column_sums_scratch(n_max, 16) + 64);
    RefineWorkspace& w = sl.ws;
    w.Y.reserve((size_t)n_max * kp_max);
    w.AY.reserve((size_t)n_max * kp_max);
    w.S4.reserve((size_t)n_max * 4);
    w.T4.reserve((size_t)n_max * 4);
    w.dev.reserve(64);
    w.part.reserve(column_sums_scratch(n_max, 16) + 64);
    w.Vd.reserve((size_t)kp_max * kp_max);
    w.Md.reserve((size_t)kp_max * kp_max);
    w.Hd.reserve((size_t)kp_max * kp_max);
    w.tb.reserve(n_max, kp_max);
    w.tb.wd.reserve((size_t)w.tb.n_pad * 128 * 2);  // W's digits at the widest projection
  }
  // the first (largest) problem on this thread: every kernel's one-time
  // attribute set-up happens before the threads start
  refine_one(B, todo[0], coeffs[todo[0]], guard, *slots[0]);
  std::atomic<size_t> next{1};
  std::vector<flz_status> status(threads, FLZ_OK);
  std::vector<std::string> message(threads);
  std::vector<int64_t> launches(threads, 0);
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t] {
      const int64_t l0 = g_kernel_launches;
      try {
        for (size_t q = next++; q < todo.size(); q = next++) refine_one(B, todo[q], coeffs[todo[q]], guard, *slots[t]);
      } catch (const Failure& f) {
        status[t] = f.status;
        message[t] = flz_last_error();
      } catch (...) {
        status[t] = FLZ_ERR_CUDA;
        message[t] = "refinement thread failed";
      }
      launches[t] = g_kernel_launches - l0;
    });
  for (auto& th : pool) th.join();
  for (int t = 0; t < threads; ++t) g_kernel_launches += launches[t];
  for (int t = 0; t < threads; ++t)
    if (status[t] != FLZ_OK) fail(status[t], "%s", message[t].c_str());
}

template <int R>
void batch_solve_r(flz_batch* B, cudaStream_t st) {
  const int count = B->count;
  const flz_params& p = B->p;
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t launches0 = g_kernel_launches;
  B->stats.assign(count, flz_stats{});
  B->evals.assign(count, {});
  B->resid.assign(count, {});
  B->evecs.clear();
  for (int i = 0; i < count; ++i) B->evecs.emplace_back(new DevBuf<double>());
  std::vector<int> act(count, 1);

  // ---- bounds: lockstep block Lanczos on A itself (degree-1 "filter" p(z) = z, c = 0, e = 1)
  {
    // at least 15 block steps (see estimate_bounds), within the smallest problem
    int64_t nmin = B->off[1] - B->off[0];
    for (int i = 1; i < count; ++i) nmin = std::min<int64_t>(nmin, B->off[i + 1] - B->off[i]);
    const int nbk = (int)std::max<int64_t>(2, std::min<int64_t>(std::max(15, (p.bounds_steps + R - 1) / R), nmin / R - 1));
    BatchEngine E;
    E.setup(B, R, nbk + 1, FLZ_PREC_FP64, st);
    E.set_active(act);
    E.set_filter(std::vector<double>(count, 0.0), std::vector<double>(count, 1.0),
                 std::vector<std::vector<double>>(count, std::vector<double>{0.0, 1.0}));
    E.start_block<R>(p.seed * 7919u + 17u);
    run_lockstep<R>(E, nbk);
    std::vector<double> Dh((size_t)count * E.nbmax * R * R), Sh(Dh.size());
    FLZ_CUDA(cudaMemcpyAsync(Dh.data(), E.Dh.p, sizeof(double) * Dh.size(), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaMemcpyAsync(Sh.data(), E.Sh.p, sizeof(double) * Sh.size(), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    parallel_for(count, [&](int i) {
      const int K = nbk * R;
      std::vector<double> T = assemble_T(Dh, Sh, i, nbk, R, E.nbmax), th, Y;
      band_eigenvalues(T, K, R, th);
      band_eigenvectors(T, K, R, th, {0, K - 1}, Y, p.seed);
      const double* S = &Sh[((size_t)i * E.nbmax + nbk - 1) * R * R];
      auto rb = [&](int t) {
        double s2 = 0.0;
        for (int a = 0; a < R; ++a) {
          double v = 0.0;
          for (int q = 0; q < R; ++q) v += S[a * R + q] * Y[(size_t)t * K + (size_t)(nbk - 1) * R + q];
          s2 += v * v;
        }
        return std::sqrt(s2);
      };
      double lo = th[0] - rb(0), hi = th[K - 1] + rb(1);
      const double margin = 1e-10 * std::max(1.0, hi - lo);
      lo = std::max(lo - margin, B->mats[i]->glo);
      hi = std::min(hi + margin, B->mats[i]->ghi);
      if (!(lo < hi)) {
        lo = B->mats[i]->glo;
        hi = B->mats[i]->ghi;
      }
      B->stats[i].lmin = lo;
      B->stats[i].lmax = hi;
    });
  }
  const double ms_bounds = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();

  // ---- per-problem map, degree, coefficients
  std::vector<double> cvec(count), evec(count);
  std::vector<std::vector<double>> coeffs(count);
  for (int i = 0; i < count; ++i) {
    flz_stats& s = B->stats[i];
    s.block_size = R;
    s.ms_bounds = ms_bounds;
    // emptiness by the Gershgorin interval; an estimate that missed an extreme
    // eigenvalue is widened to cover the interval (as in the single solver)
    const flz_matrix* Ai = B->mats[i];
    if (B->beta[i] < Ai->glo || B->alpha[i] > Ai->ghi)
      fail(FLZ_ERR_EMPTY_INTERVAL, "problem %d: [%g, %g] misses the Gershgorin interval [%g, %g]", i, B->alpha[i],
           B->beta[i], Ai->glo, Ai->ghi);
    if (B->beta[i] < s.lmin) s.lmin = std::max(B->alpha[i], Ai->glo);
    if (B->alpha[i] > s.lmax) s.lmax = std::min(B->beta[i], Ai->ghi);
    const double c = 0.5 * (s.lmin + s.lmax), e = 0.5 * (s.lmax - s.lmin);
    double am = (B->alpha[i] - c) / e, bm = (B->beta[i] - c) / e;
    am = std::max(am, -1.0);
    bm = std::min(bm, 1.0);
    const int m = p.degree > 0 ? p.degree : auto_degree(am, bm, p.degree_eps, p.max_degree);
    if (m < 1) fail(FLZ_ERR_CAPACITY, "problem %d: no degree <= %d meets the degree rule", i, p.max_degree);
    coeffs[i].resize(m + 1);
    filter_coeffs_for(p, am, bm, m, coeffs[i].data());
    s.c = c;
    s.e = e;
    s.alpha_mapped = am;
    s.beta_mapped = bm;
    s.degree = m;
    cvec[i] = c;
    evec[i] = e;
  }

  // ---- main phase
  int64_t nmax_rows = 0;
  for (int i = 0; i < count; ++i) nmax_rows = std::max<int64_t>(nmax_rows, B->off[i + 1] - B->off[i]);
  int64_t kcap = p.max_basis > 0 ? p.max_basis : 2000;
  size_t free_b = 0, total_b = 0;
  FLZ_CUDA(cudaMemGetInfo(&free_b, &total_b));
  kcap = std::min<int64_t>(kcap, (int64_t)(0.5 * (double)free_b / (8.0 * (double)B->N)));
  kcap = std::min<int64_t>(kcap, nmax_rows);
  // Tensor-core reorthogonalization unless the CUDA cores are asked for: the
  // digit copies (16 bytes per value, grown with the basis) and the FP64
  // basis share 60 % of the free memory; AUTO keeps the CUDA cores where
  // that would shrink the basis below 200 vectors per problem.
  const int64_t kcap_tc = (int64_t)(0.6 * (double)free_b / (24.0 * (double)B->N));
  const bool use_tc = p.ortho == FLZ_ORTHO_TENSOR || (p.ortho == FLZ_ORTHO_AUTO && std::min(kcap, kcap_tc) >= 200);
  if (use_tc) kcap = std::max<int64_t>(2 * R, std::min(kcap, kcap_tc));
  const int nbmax = (int)std::max<int64_t>(2, kcap / R);
  BatchEngine E;
  E.setup(B, R, nbmax, p.precision, st);
  E.set_active(act);
  E.set_filter(cvec, evec, coeffs);
  for (int i = 0; i < count; ++i) {
    B->stats[i].filter_precision = E.precision;
    B->stats[i].ortho = use_tc ? FLZ_ORTHO_TENSOR : FLZ_ORTHO_CUDA_CORES;
  }
  E.start_block<R>(p.seed);
  if (use_tc) {
    E.setup_tc(16 * R);
    E.tc_append(0, act);
  }

  const int guard = p.guard > 0 ? p.guard : std::max(R, 3);
  // With refinement (reduced-precision filter) the lockstep phase stops at the
  // filter's floor and each problem's pairs are then refined to p.tol.
  const bool refining = p.refine == 1 && (E.precision == FLZ_PREC_FP32 || E.precision == FLZ_PREC_BF16);
  const double tol = refining ? std::max(p.tol, E.precision == FLZ_PREC_FP32 ? 1e-5 : 1e-2) : p.tol;
  std::vector<int64_t> prev_count(count, -1);
  std::vector<int> gate_len(count, 16), iters(count, 0), checks(count, 0);
  std::vector<int> converged(count, 0);
  DevBuf<double> X, AX, Ytab, lam, sums, cpart;
  X.reserve((size_t)B->N * 16);
  AX.reserve((size_t)B->N * 16);
  lam.reserve((size_t)count * 16);
  sums.reserve((size_t)count * 16 * 3);
  cpart.reserve((size_t)E.n_chunks * 16);
  DevBuf<int> walking;
  walking.reserve(count);
  std::vector<std::vector<double>> found_vals(count), found_res(count);
  std::vector<int64_t> found(count, 0);

  int k = 0;
  double ms_steps = 0.0, ms_check = 0.0;
  // graph of one step (CUDA-core reorthogonalization), or of its two halves
  // around the per-problem tensor-core CGS2, replayed between checks
  const int64_t before_capture = g_kernel_launches;
  struct GraphGuard {
    cudaGraphExec_t g = nullptr;
    ~GraphGuard() {
      if (g) cudaGraphExecDestroy(g);
    }
  } graph_a, graph_b;
  // the persistent filter (one cooperative launch per step) is captured too
  // where stream capture takes a cooperative launch; otherwise it is launched
  // directly each step
  E.persistent = p.persistent == 1 && E.precision == FLZ_PREC_FX64;
  bool direct_filter = false;
  if (E.persistent) {
    const int64_t before_a = g_kernel_launches;
    try {
      graph_a.g = capture_part(E, [&] { E.apply_filter<R>(); });
    } catch (const Failure&) {
      cudaGetLastError();
      clear_last_error();
      g_kernel_launches = before_a;  // launches of the abandoned capture
      graph_a.g = nullptr;
      direct_filter = true;
    }
    graph_b.g = capture_part(E, [&] {
      if (use_tc) E.step_tail<R>();
      else E.step_after_filter<R>();
    });
  } else if (use_tc) {
    graph_a.g = capture_part(E, [&] { E.apply_filter<R>(); });
    graph_b.g = capture_part(E, [&] { E.step_tail<R>(); });
  } else {
    graph_a.g = capture_part(E, [&] { E.step<R>(); });
  }
  const bool split = use_tc || E.persistent;  // filter and the rest in separate graphs
  const int64_t launches_per_step = g_kernel_launches - before_capture;
  g_kernel_launches = before_capture;  // captured, not launched
  while (k < nbmax) {
    const auto ts = std::chrono::steady_clock::now();
    const int todo = std::min(p.check_every - (k % p.check_every), nbmax - k);
    for (int s = 0; s < todo; ++s) {
      if (direct_filter) E.apply_filter<R>();
      else FLZ_CUDA(cudaGraphLaunch(graph_a.g, st));
      if (use_tc) {
        E.tc_orth((k + s + 1) * R, act);  // the basis holds Q_0 .. Q_j, j = k + s
        FLZ_CUDA(cudaGraphLaunch(graph_b.g, st));
        E.tc_append((k + s + 1) * R, act);
      } else if (split) {
        FLZ_CUDA(cudaGraphLaunch(graph_b.g, st));
      }
    }
    g_kernel_launches += (int64_t)todo * launches_per_step;
    k += todo;
    FLZ_CUDA(cudaStreamSynchronize(st));
    if (use_tc) E.tc_check();
    ms_steps += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    const bool last = k >= nbmax;
    const auto tc = std::chrono::steady_clock::now();
    int hfail = 0;
    FLZ_CUDA(cudaMemcpy(&hfail, E.fail.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (E.precision == FLZ_PREC_FX64) fx_batch_check_flag(B->fxb, st);
    std::vector<double> Dh((size_t)count * nbmax * R * R), Sh(Dh.size());
    FLZ_CUDA(cudaMemcpy(Dh.data(), E.Dh.p, sizeof(double) * Dh.size(), cudaMemcpyDeviceToHost));
    FLZ_CUDA(cudaMemcpy(Sh.data(), E.Sh.p, sizeof(double) * Sh.size(), cudaMemcpyDeviceToHost));
    const int K = k * R;
    std::vector<WalkState> ws(count);
    std::vector<int> walk_flag(count, 0);
    parallel_for(count, [&](int i) {
      if (!act[i]) return;
      WalkState& w = ws[i];
      checks[i]++;
      iters[i] = k;
      w.K = K;
      w.T = assemble_T(Dh, Sh, i, k, R, nbmax);
      band_eigenvalues(w.T, K, R, w.theta);
      w.order.resize(K);
      for (int q = 0; q < K; ++q) w.order[q] = K - 1 - q;
      const int m = B->stats[i].degree;
      const double anorm = std::max(std::fabs(B->stats[i].lmin), std::fabs(B->stats[i].lmax));
      const bool fp64_class = E.precision == FLZ_PREC_FP64 || E.precision == FLZ_PREC_FX64;
      const double p_gate = std::min(fp64_class ? 1e-2 : 1e-1,
                                     10.0 * 1.1 * (double)m * m * tol * anorm / B->stats[i].e);
      const int g_cnt = std::min(gate_len[i], K);
      const double* S = &Sh[((size_t)i * nbmax + k - 1) * R * R];
      for (int g0 = 0; g0 < g_cnt && w.all_small; g0 += 8) {
        std::vector<int> gidx(w.order.begin() + g0, w.order.begin() + std::min(g_cnt, g0 + 8));
        std::vector<double> Yg;
        band_eigenvectors(w.T, K, R, w.theta, gidx, Yg, p.seed + (uint64_t)g0);
        for (size_t t = 0; t < gidx.size() && w.all_small; ++t) {
          double s2 = 0.0;
          for (int a = 0; a < R; ++a) {
            double v = 0.0;
            for (int q = 0; q < R; ++q) v += S[a * R + q] * Yg[t * K + (size_t)(k - 1) * R + q];
            s2 += v * v;
          }
          if (!(std::sqrt(s2) <= p_gate)) w.all_small = false;
        }
      }
      walk_flag[i] = w.all_small ? 1 : 0;
      found_vals[i].clear();
      found_res[i].clear();
      found[i] = 0;
    });
    // walk in rounds of 16 Ritz pairs for every problem still walking
    for (int pos = 0;; pos += 16) {
      bool any = false;
      for (int i = 0; i < count; ++i) any |= walk_flag[i] != 0;
      if (!any || pos >= K) break;
      std::vector<double> tab((size_t)count * K * 16, 0.0);
      std::vector<int> cnts(count, 0);
      parallel_for(count, [&](int i) {
        if (!walk_flag[i]) return;
        WalkState& w = ws[i];
        const int cnt = std::min(16, K - pos);
        cnts[i] = cnt;
        // kept orthogonal to the earlier chunks' vectors of nearby eigenvalues
        // (copies of a multiple eigenvalue may straddle two chunks)
        std::vector<int> idx(w.order.begin() + pos, w.order.begin() + pos + cnt);
        std::vector<double> Y;
        band_eigenvectors(w.T, K, R, w.theta, idx, Y, p.seed, &w.walkY, &w.walkIdx);
        w.walkY.insert(w.walkY.end(), Y.begin(), Y.end());
        w.walkIdx.insert(w.walkIdx.end(), idx.begin(), idx.end());
        for (int t = 0; t < cnt; ++t)
          for (int q = 0; q < K; ++q) tab[((size_t)i * K + q) * 16 + t] = Y[(size_t)t * K + q];
      });
      Ytab.reserve(tab.size());
      FLZ_CUDA(cudaMemcpyAsync(Ytab.p, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st));
      FLZ_CUDA(cudaMemcpyAsync(walking.p, walk_flag.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
      if (use_tc) {
        E.on_side_streams(walk_flag, [&](int i, cudaStream_t s) {
          E.tcb[i]->multiply(K, Ytab.p + (size_t)i * K * 16, 16, 16, X.p + (size_t)B->off[i] * 16, 16, s);
        });
      } else {
        E.update<16>(E.Q.p, k, R, Ytab.p, (long long)K * 16, 1.0, 0.0, X.p, 16, walking.p);
      }
      seg_spmm_kernel<<<(unsigned)(((B->N + 1) / 2 * 32 + 255) / 256), 256, 0, st>>>(B->N, 16, 16, B->rowptr.p, B->col.p,
                                                                              B->val.p, X.p, AX.p);
      FLZ_LAUNCH_CHECK();
      seg_colsum_kernel<<<E.n_chunks, kT, 0, st>>>(X.p, X.p, nullptr, 0, B->d_c_row0.p, B->d_c_row1.p, B->d_c_mat.p, walking.p, cpart.p);
      FLZ_LAUNCH_CHECK();
      seg_colsum_reduce_kernel<<<gsb((long long)count * 16), 256, 0, st>>>(count, B->d_c_beg.p, walking.p, cpart.p, sums.p);
      FLZ_LAUNCH_CHECK();
      seg_colsum_kernel<<<E.n_chunks, kT, 0, st>>>(X.p, AX.p, nullptr, 0, B->d_c_row0.p, B->d_c_row1.p, B->d_c_mat.p, walking.p, cpart.p);
      FLZ_LAUNCH_CHECK();
      seg_colsum_reduce_kernel<<<gsb((long long)count * 16), 256, 0, st>>>(count, B->d_c_beg.p, walking.p, cpart.p, sums.p + count * 16);
      FLZ_LAUNCH_CHECK();
      std::vector<double> hs((size_t)count * 32);
      FLZ_CUDA(cudaMemcpyAsync(hs.data(), sums.p, sizeof(double) * count * 32, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaStreamSynchronize(st));
      std::vector<double> hl((size_t)count * 16, 0.0);
      for (int i = 0; i < count; ++i)
        for (int t = 0; t < 16; ++t) {
          const double xx = hs[(size_t)i * 16 + t];
          hl[(size_t)i * 16 + t] = xx > 0 ? hs[(size_t)count * 16 + i * 16 + t] / xx : 0.0;
        }
      FLZ_CUDA(cudaMemcpyAsync(lam.p, hl.data(), sizeof(double) * hl.size(), cudaMemcpyHostToDevice, st));
      seg_colsum_kernel<<<E.n_chunks, kT, 0, st>>>(X.p, AX.p, lam.p, 1, B->d_c_row0.p, B->d_c_row1.p, B->d_c_mat.p, walking.p, cpart.p);
      FLZ_LAUNCH_CHECK();
      seg_colsum_reduce_kernel<<<gsb((long long)count * 16), 256, 0, st>>>(count, B->d_c_beg.p, walking.p, cpart.p, sums.p + 2 * count * 16);
      FLZ_LAUNCH_CHECK();
      std::vector<double> hr((size_t)count * 16);
      FLZ_CUDA(cudaMemcpyAsync(hr.data(), sums.p + 2 * count * 16, sizeof(double) * count * 16, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaStreamSynchronize(st));
      for (int i = 0; i < count; ++i) {
        if (!walk_flag[i]) continue;
        WalkState& w = ws[i];
        const int n_i = B->off[i + 1] - B->off[i];
        const double anorm = std::max(std::fabs(B->stats[i].lmin), std::fabs(B->stats[i].lmax));
        for (int t = 0; t < cnts[i] && !w.done; ++t) {
          ++w.walked;
          const double xx = hs[(size_t)i * 16 + t];
          const double l = hl[(size_t)i * 16 + t];
          const double res = std::sqrt(std::max(hr[(size_t)i * 16 + t], 0.0) / std::max(xx, 1e-300)) / anorm;
          if (!(res <= tol)) {
            w.all_small = false;
            w.done = true;
            break;
          }
          if (l >= B->alpha[i] && l <= B->beta[i]) {
            auto& buf = *B->evecs[i];
            const size_t need = (size_t)(found[i] + 1) * n_i;
            if (buf.count < need) {
              DevBuf<double> grown;
              grown.reserve(std::max(need, buf.count * 2));
              if (found[i] > 0)
                FLZ_CUDA(cudaMemcpyAsync(grown.p, buf.p, sizeof(double) * found[i] * n_i, cudaMemcpyDeviceToDevice, st));
              FLZ_CUDA(cudaStreamSynchronize(st));
              std::swap(grown.p, buf.p);
              std::swap(grown.count, buf.count);
            }
            // the unit eigenvector, in one launch with no host round trip
            rows_to_columns(X.p + (size_t)B->off[i] * 16 + t, n_i, 1, 16, buf.p + (size_t)found[i] * n_i, n_i, st,
                            1.0 / std::sqrt(xx));
            found_vals[i].push_back(l);
            found_res[i].push_back(res);
            ++found[i];
            ++w.inside;
          } else {
            ++w.outside;
            if (w.outside >= guard) {
              w.done = true;
              break;
            }
          }
        }
        if (!w.done && pos + cnts[i] >= K) w.done = true;
        if (w.done) walk_flag[i] = 0;
      }
    }
    for (int i = 0; i < count; ++i) {
      if (!act[i]) continue;
      WalkState& w = ws[i];
      if (w.walked > 0) gate_len[i] = std::max(16, w.walked);
      const bool complete = w.all_small && w.outside >= guard;
      const bool conv = complete && prev_count[i] >= 0 && w.inside == prev_count[i];
      prev_count[i] = complete ? w.inside : -1;
      // a problem whose Krylov space would outgrow its dimension stops here
      const bool exhausted = (int64_t)(k + p.check_every) * R > (int64_t)(B->off[i + 1] - B->off[i]);
      if (conv || last || exhausted) {
        converged[i] = conv ? 1 : 0;
        act[i] = 0;
        // results: ascending eigenvalues (columns permuted accordingly)
        const int n_i = B->off[i + 1] - B->off[i];
        const int64_t f = found[i];
        std::vector<int> perm(f);
        for (int q = 0; q < f; ++q) perm[q] = q;
        std::sort(perm.begin(), perm.end(), [&](int a, int b) { return found_vals[i][a] < found_vals[i][b]; });
        if (f > 0) {
          DevBuf<double> tmp;
          tmp.reserve((size_t)f * n_i);
          for (int q = 0; q < f; ++q)
            FLZ_CUDA(cudaMemcpyAsync(tmp.p + (size_t)q * n_i, B->evecs[i]->p + (size_t)perm[q] * n_i, sizeof(double) * n_i,
                                     cudaMemcpyDeviceToDevice, st));
          FLZ_CUDA(cudaStreamSynchronize(st));
          std::swap(tmp.p, B->evecs[i]->p);
          std::swap(tmp.count, B->evecs[i]->count);
        }
        B->evals[i].resize(f);
        B->resid[i].resize(f);
        double maxres = 0.0;
        for (int q = 0; q < f; ++q) {
          B->evals[i][q] = found_vals[i][perm[q]];
          B->resid[i][q] = found_res[i][perm[q]];
          maxres = std::max(maxres, B->resid[i][q]);
        }
        flz_stats& s = B->stats[i];
        s.iters = k;
        s.matvecs = (int64_t)R * s.degree * k;
        s.count = f;
        s.converged = converged[i];
        s.checks = checks[i];
        s.max_residual = maxres;
        s.basis_vectors = (int64_t)k * R;
      }
    }
    E.set_active(act);
    ms_check += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc).count();
    bool any = false;
    for (int i = 0; i < count; ++i) any |= act[i] != 0;
    if (!any) break;
    if (hfail) {
      // a Cholesky pivot failed even with the shift: the block is numerically
      // rank deficient; continuing is still safe (the factor was regularized)
      FLZ_CUDA(cudaMemsetAsync(E.fail.p, 0, sizeof(int), st));
    }
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
  if (refining) refine_problems(B, coeffs, converged, guard);
  const double total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < count; ++i) {
    B->stats[i].ms_filter = ms_steps;  // the lockstep steps (filter + orthogonalization) of the whole batch
    B->stats[i].ms_check = ms_check;
    B->stats[i].ms_total = total;
    B->stats[i].kernel_launches = g_kernel_launches - launches0;
    B->stats[i].tile_rows = E.precision == FLZ_PREC_FX64 ? B->fxb.rows : 0;
  }
  B->solved = true;
}

}  // namespace

int batch_autotune(flz_batch* B, cudaStream_t st);
void tune_rows(flz_batch* B, int r, double t256, cudaStream_t st);

flz_status batch_solve(flz_batch* B, cudaStream_t user) {
  // Work runs on a private non-blocking stream (graphs cannot be captured on
  // the legacy default stream), ordered after the caller's stream.
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  FLZ_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    cudaEvent_t e;
    ~StreamGuard() {
      if (s) cudaStreamSynchronize(s), cudaStreamDestroy(s);
      if (e) cudaEventDestroy(e);
    }
  } guard{st, nullptr};
  FLZ_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  guard.e = ev;
  FLZ_CUDA(cudaEventRecord(ev, user));
  FLZ_CUDA(cudaStreamWaitEvent(st, ev, 0));
  // tuned on the handle's first solve; later solves reuse the choice
  int r = B->p.block_size;
  if (B->tuned_rows == 0 || (r == 0 && B->tuned_r == 0)) {
    if (r == 0) B->tuned_r = batch_autotune(B, st);
    else tune_rows(B, r, 0.0, st);
    B->tuned_rows = B->fxb.rows;
  }
  if (r == 0) r = B->tuned_r;
  B->fxb.rows = B->tuned_rows;
  B->r = r;
  FLZ_DISPATCH_R(r, batch_solve_r, B, st);
  FLZ_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < B->count; ++i)
    if (!B->stats[i].converged) return FLZ_ERR_NOT_CONVERGED;
  return FLZ_OK;
}

// Filter timings of the concatenated matrix at block width r and, for the
// fixed-point filter, `rows` rows per CTA: the time of a degree-16
// application minus that of a degree-8 one (each the best of three after a
// warm-up), i.e. of 8 middle degree steps, the steps that dominate a solve.
// Returns ms per vector and degree step.
double time_filter_degree(flz_batch* B, int r, int rows, int degree, cudaStream_t st);
double time_filter(flz_batch* B, int r, int rows, cudaStream_t st) {
  const double t16 = time_filter_degree(B, r, rows, 16, st);
  const double t8 = time_filter_degree(B, r, rows, 8, st);
  return std::max(t16 - t8, 1e-9) / 8.0;
}
double time_filter_degree(flz_batch* B, int r, int rows, int degree, cudaStream_t st) {
  cudaEvent_t e0, e1;
  FLZ_CUDA(cudaEventCreate(&e0));
  FLZ_CUDA(cudaEventCreate(&e1));
  BatchEngine E;
  E.setup(B, r, 2, B->p.precision, st);
  std::vector<int> act(B->count, 1);
  E.set_active(act);
  std::vector<double> probe(degree + 1, 0.0);
  probe[degree] = 1.0;
  E.set_filter(std::vector<double>(B->count, 0.0), std::vector<double>(B->count, 1e6),
               std::vector<std::vector<double>>(B->count, probe));
  B->fxb.rows = rows;
  FLZ_CUDA(cudaMemsetAsync(E.Q.p, 0, sizeof(double) * B->N * r, st));
  FLZ_CUDA(cudaMemsetAsync(E.jdev.p, 0, sizeof(int), st));
  auto run = [&] {
    switch (r) {
      case 4: E.apply_filter<4>(); break;
      case 8: E.apply_filter<8>(); break;
      default: E.apply_filter<16>(); break;
    }
  };
  run();
  float best = 1e30f;
  for (int q = 0; q < 3; ++q) {
    FLZ_CUDA(cudaEventRecord(e0, st));
    run();
    FLZ_CUDA(cudaEventRecord(e1, st));
    FLZ_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FLZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best / r;
}

// The fixed-point filter's tile shape at width r (t256: its time_filter at
// 256 rows per CTA, if already measured): 128 rows per CTA only if that is at least 5 %
// faster (near-equal timings must not flip the choice from run to run), else
// 256. A tile shape the caller fixed is kept.
void tune_rows(flz_batch* B, int r, double t256, cudaStream_t st) {
  if (B->p.tile_rows != 0) {
    B->fxb.rows = B->p.tile_rows;
    return;
  }
  B->fxb.rows = 256;
  if (B->p.precision != FLZ_PREC_FX64) return;
  if (t256 <= 0.0) t256 = time_filter(B, r, 256, st);
  const double t128 = time_filter(B, r, 128, st);
  B->fxb.rows = t128 < 0.95 * t256 ? 128 : 256;
}

// Picks r in {4, 8, 16} (at 256 rows per CTA, or the caller's tile shape),
// then the fixed-point filter's rows per CTA at that r: a wider block is
// taken only if it is at least 25 % cheaper per vector than the current
// choice (a wider block reaches a lower Krylov degree within the same basis
// capacity, and near-equal timings must not flip the choice from run to run).
int batch_autotune(flz_batch* B, cudaStream_t st) {
  double best = 1e300;
  int best_r = 4;
  const int rows0 = B->p.tile_rows != 0 ? B->p.tile_rows : 256;
  for (int r : {4, 8, 16}) {
    const double per_vec = time_filter(B, r, rows0, st);
    if (per_vec < 0.75 * best) {
      best = per_vec;
      best_r = r;
    }
  }
  tune_rows(B, best_r, best, st);
  return best_r;
}

}  // namespace flz

// ---- C ABI ---------------------------------------------------------------------

using flz::fail;

extern "C" {

flz_status flz_batch_create(int32_t count, flz_matrix* const* mats, const double* alphas, const double* betas,
                            const flz_params* params, flz_batch** out) {
  FLZ_API_BEGIN
  if (!out || !mats || !alphas || !betas || count < 1 || count > flz::kMaxProblems)
    fail(FLZ_ERR_INVALID_ARG, "need 1 <= count <= %d and non-null arrays", flz::kMaxProblems);
  *out = nullptr;
  flz_params p;
  if (params) p = *params;
  else flz_params_default(&p);
  if (!(p.block_size == 0 || p.block_size == 1 || p.block_size == 2 || p.block_size == 4 || p.block_size == 8 ||
        p.block_size == 16))
    fail(FLZ_ERR_INVALID_ARG, "batch block_size must be 0 (autotune) or one of 1, 2, 4, 8, 16");
  if (p.degree < 0 || p.max_degree < 1 || p.check_every < 1 || !(p.tol > 0.0) || p.bounds_steps < 1 ||
      p.damping < 0 || p.damping > 2 || !(p.transition >= 0.0) || p.persistent < 0 || p.persistent > 1 || p.refine < 0 || p.refine > 1 ||
      (p.tile_rows != 0 && p.tile_rows != 128 && p.tile_rows != 256))
    fail(FLZ_ERR_INVALID_ARG, "invalid parameter");
  if (p.recurrence != FLZ_REC_FORWARD) fail(FLZ_ERR_INVALID_ARG, "batches use the forward recurrence only");
  if (p.precision < FLZ_PREC_FP64 || p.precision > FLZ_PREC_FX64)
    fail(FLZ_ERR_INVALID_ARG, "batches support the FP64, FP32, BF16, double-FP32 and fixed-point filters");
  std::unique_ptr<flz_batch> B(new flz_batch());
  B->count = count;
  B->p = p;
  B->off.assign(count + 1, 0);
  int64_t nnz = 0;
  for (int i = 0; i < count; ++i) {
    if (!mats[i]) fail(FLZ_ERR_INVALID_ARG, "matrix %d is NULL", i);
    if (!(alphas[i] < betas[i])) fail(FLZ_ERR_INVALID_ARG, "problem %d: need alpha < beta", i);
    B->mats.push_back(mats[i]);
    B->alpha.push_back(alphas[i]);
    B->beta.push_back(betas[i]);
    if ((int64_t)B->off[i] + mats[i]->n > 2147483647LL) fail(FLZ_ERR_INVALID_ARG, "total rows exceed int32");
    B->off[i + 1] = B->off[i] + (int)mats[i]->n;
    nnz += mats[i]->nnz;
    B->max_row_nnz = std::max(B->max_row_nnz, mats[i]->max_row_nnz);
  }
  if (nnz > 2147483647LL) fail(FLZ_ERR_INVALID_ARG, "total nnz exceeds int32");
  B->N = B->off[count];
  B->nnz = nnz;
  B->rowptr.reserve((size_t)B->N + 1);
  B->col.reserve((size_t)nnz);
  B->val.reserve((size_t)nnz);
  B->diag_pos.reserve((size_t)B->N);
  int64_t nz0 = 0;
  for (int i = 0; i < count; ++i) {
    flz_matrix* A = mats[i];
    flz::offset_copy_kernel<<<flz::gsb(A->n + 1), 256>>>(A->rowptr.p, B->rowptr.p + B->off[i], A->n + 1, (int)nz0);
    FLZ_LAUNCH_CHECK();
    flz::offset_copy_kernel<<<flz::gsb(A->nnz), 256>>>(A->col.p, B->col.p + nz0, A->nnz, B->off[i]);
    FLZ_LAUNCH_CHECK();
    flz::offset_copy_kernel<<<flz::gsb(A->n), 256>>>(A->diag_pos.p, B->diag_pos.p + B->off[i], A->n, (int)nz0);
    FLZ_LAUNCH_CHECK();
    FLZ_CUDA(cudaMemcpy(B->val.p + nz0, A->val.p, sizeof(double) * A->nnz, cudaMemcpyDeviceToDevice));
    nz0 += A->nnz;
  }
  FLZ_CUDA(cudaDeviceSynchronize());
  FLZ_CUDA(cudaMalloc(reinterpret_cast<void**>(&B->d_off.p), sizeof(int) * (count + 1)));
  B->d_off.count = count + 1;
  FLZ_CUDA(cudaMemcpy(B->d_off.p, B->off.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice));
  // max nnz over 256-row blocks of the concatenated matrix
  {
    flz_matrix tmp;
    tmp.n = B->N;
    tmp.rowptr.p = B->rowptr.p;
    B->max_cta_nnz = flz::max_block_nnz(&tmp, 256);
    tmp.rowptr.p = nullptr;
  }
  flz::build_chunks(B.get());
  *out = B.release();
  FLZ_API_END
}

flz_status flz_batch_destroy(flz_batch* b) {
  FLZ_API_BEGIN
  delete b;
  FLZ_API_END
}

flz_status flz_batch_solve(flz_batch* b, void* stream) {
  flz::clear_last_error();
  try {
    if (!b) fail(FLZ_ERR_INVALID_ARG, "batch is NULL");
    const flz_status st = flz::batch_solve(b, static_cast<cudaStream_t>(stream));
    if (st == FLZ_ERR_NOT_CONVERGED) flz::set_last_error("some problems reached the basis capacity first");
    return st;
  } catch (const flz::Failure& f) {
    return f.status;
  } catch (...) {
    flz::set_last_error("unexpected internal error");
    return FLZ_ERR_CUDA;
  }
}

static const flz_batch* checked(const flz_batch* b, int32_t index) {
  if (!b) fail(FLZ_ERR_INVALID_ARG, "batch is NULL");
  if (index < 0 || index >= b->count) fail(FLZ_ERR_INVALID_ARG, "index %d out of range", index);
  if (!b->solved) fail(FLZ_ERR_NOT_SOLVED, "no solve yet");
  return b;
}

flz_status flz_batch_get_count(const flz_batch* b, int32_t index, int64_t* count) {
  FLZ_API_BEGIN
  checked(b, index);
  if (!count) fail(FLZ_ERR_INVALID_ARG, "count is NULL");
  *count = (int64_t)b->evals[index].size();
  FLZ_API_END
}

flz_status flz_batch_get_eigenvalues(const flz_batch* b, int32_t index, double* out, int64_t cap) {
  FLZ_API_BEGIN
  checked(b, index);
  const auto& v = b->evals[index];
  if (cap < (int64_t)v.size()) fail(FLZ_ERR_CAPACITY, "need %zu slots", v.size());
  if (!v.empty() && !out) fail(FLZ_ERR_INVALID_ARG, "out is NULL");
  std::copy(v.begin(), v.end(), out);
  FLZ_API_END
}

flz_status flz_batch_get_residuals(const flz_batch* b, int32_t index, double* out, int64_t cap) {
  FLZ_API_BEGIN
  checked(b, index);
  const auto& v = b->resid[index];
  if (cap < (int64_t)v.size()) fail(FLZ_ERR_CAPACITY, "need %zu slots", v.size());
  if (!v.empty() && !out) fail(FLZ_ERR_INVALID_ARG, "out is NULL");
  std::copy(v.begin(), v.end(), out);
  FLZ_API_END
}

flz_status flz_batch_get_eigenvectors(const flz_batch* b, int32_t index, double* out, int64_t ld, int64_t cap_cols,
                                      flz_memspace where) {
  FLZ_API_BEGIN
  checked(b, index);
  const int64_t n = b->off[index + 1] - b->off[index];
  const int64_t cnt = (int64_t)b->evals[index].size();
  if (ld < n) fail(FLZ_ERR_INVALID_ARG, "ld < n");
  if (cap_cols < cnt) fail(FLZ_ERR_CAPACITY, "need %lld columns", (long long)cnt);
  if (where != FLZ_HOST && where != FLZ_DEVICE) fail(FLZ_ERR_INVALID_ARG, "bad memspace");
  if (cnt == 0) return FLZ_OK;
  if (!out) fail(FLZ_ERR_INVALID_ARG, "out is NULL");
  FLZ_CUDA(cudaMemcpy2D(out, sizeof(double) * ld, b->evecs[index]->p, sizeof(double) * n, sizeof(double) * n,
                        (size_t)cnt, where == FLZ_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
  FLZ_API_END
}

flz_status flz_batch_get_stats(const flz_batch* b, int32_t index, flz_stats* out) {
  FLZ_API_BEGIN
  checked(b, index);
  if (!out) fail(FLZ_ERR_INVALID_ARG, "out is NULL");
  *out = b->stats[index];
  FLZ_API_END
}

}  // extern "C"
