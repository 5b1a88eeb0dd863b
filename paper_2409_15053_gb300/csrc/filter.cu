// The hot path: W = p_m(Ahat) V with Ahat = (A - cI)/e (eq. transf) and
// p_m = sum_{i<=m} b_i T_i (Section 2.2).
//
// The paper evaluates p_m(Ahat)V with a vectorized Clenshaw recurrence built
// from library SpMV calls (Section 2.2, 3.2). Here the forward three-term
// Chebyshev recurrence (eq. def:cheb1) is fused with the running sum, so one
// launch per degree makes exactly one pass over the CSR matrix and the vector
// streams:
//   step 0   Y_1 = Ahat V,                         acc  = b_0 V + b_1 Y_1
//   step k   Y_{k+1} = 2 Ahat Y_k - Y_{k-1},       acc += b_{k+1} Y_{k+1}
// written as Y_next = alpha (A Y_cur) + beta Y_cur - gamma Y_prev with
// (alpha, beta, gamma) = (1/e, -c/e, 0) at step 0 and (2/e, -2c/e, 1) after.
//
// Thread mapping: r consecutive lanes own one row (lane c computes column c),
// 32/r rows per warp. Vectors are n x r row-major so one gathered row Y[col]
// is r contiguous elements (one 32-byte sector for r = 4 in FP64). The CSR
// index/value loads of a row are shared by its r lanes (same address, one
// transaction). Y_{k-1} is overwritten in place by Y_{k+1}.
#include "flz_internal.h"

namespace flz {

namespace {

template <class S>
struct Arith {
  using type = float;
};
template <>
struct Arith<double> {
  using type = double;
};

__device__ __forceinline__ double to_arith(double x) { return x; }
__device__ __forceinline__ float to_arith(float x) { return x; }
__device__ __forceinline__ float to_arith(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class S>
__device__ __forceinline__ S from_arith(typename Arith<S>::type x);
template <>
__device__ __forceinline__ double from_arith<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_arith<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_arith<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <class O, class A>
__device__ __forceinline__ O store_as(A x) { return static_cast<O>(x); }

constexpr int kThreads = 256;

// One fused Chebyshev degree step over the whole matrix.
//   MS: matrix value storage, VS: recurrence vector storage,
//   AccS: running-sum input storage, OutS: running-sum output storage.
// ynext may alias yprev; acc_out may alias acc_in (each element is read and
// written by the same thread).
template <class MS, class VS, class AccS, class OutS, bool FIRST>
__global__ void __launch_bounds__(kThreads) cheb_step_kernel(
    int n, int r, int rows_per_warp, const int* __restrict__ rowptr, const int* __restrict__ col,
    const MS* __restrict__ val, const VS* __restrict__ ycur, const VS* yprev, VS* ynext, const AccS* acc_in,
    OutS* acc_out, typename Arith<VS>::type alpha, typename Arith<VS>::type beta,
    typename Arith<VS>::type b_cur, typename Arith<VS>::type b_next) {
  using A = typename Arith<VS>::type;
  const int lane = threadIdx.x & 31;
  const int sub = lane / r;
  const int c = lane - sub * r;
  const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const long long row = warp * rows_per_warp + sub;
  if (sub >= rows_per_warp || row >= n) return;
  int j = __ldg(rowptr + row);
  const int jend = __ldg(rowptr + row + 1);
  A s0 = A(0), s1 = A(0);
  for (; j + 4 <= jend; j += 4) {
    const int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2), c3 = __ldg(col + j + 3);
    const A a0 = to_arith(val[j]), a1 = to_arith(val[j + 1]), a2 = to_arith(val[j + 2]), a3 = to_arith(val[j + 3]);
    const A y0 = to_arith(ycur[(size_t)c0 * r + c]);
    const A y1 = to_arith(ycur[(size_t)c1 * r + c]);
    const A y2 = to_arith(ycur[(size_t)c2 * r + c]);
    const A y3 = to_arith(ycur[(size_t)c3 * r + c]);
    s0 = fma(a0, y0, s0);
    s1 = fma(a1, y1, s1);
    s0 = fma(a2, y2, s0);
    s1 = fma(a3, y3, s1);
  }
  for (; j < jend; ++j) {
    const int cj = __ldg(col + j);
    s0 = fma(to_arith(val[j]), to_arith(ycur[(size_t)cj * r + c]), s0);
  }
  const size_t idx = (size_t)row * r + c;
  const A yc = to_arith(ycur[idx]);
  A yn = fma(alpha, s0 + s1, beta * yc);
  if (!FIRST) yn -= to_arith(yprev[idx]);
  const VS yn_s = from_arith<VS>(yn);
  ynext[idx] = yn_s;
  const A yq = to_arith(yn_s);
  A acc = FIRST ? b_cur * yc : A(to_arith(acc_in[idx]));
  acc = fma(b_next, yq, acc);
  acc_out[idx] = store_as<OutS>(acc);
}

template <class S>
__global__ void convert_kernel(const double* __restrict__ in, S* __restrict__ out, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = from_arith<S>((typename Arith<S>::type)in[i]);
}

__global__ void scale_kernel(const double* __restrict__ in, double* __restrict__ out, double s, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = s * in[i];
}

inline unsigned grid_for_rows(int64_t n, int r) {
  const int rpw = 32 / r;
  const int64_t warps = (n + rpw - 1) / rpw;
  return (unsigned)((warps * 32 + kThreads - 1) / kThreads);
}

inline unsigned grid_stride_blocks(size_t count) {
  size_t b = (count + 255) / 256;
  return (unsigned)std::min<size_t>(b, 152 * 16);
}

template <class MS, class VS, class AccT>
void run_recurrence(const flz_matrix* A, const MS* val, double c, double e, const double* b, int m, int r,
                    const VS* v, VS* ya, VS* yb, AccT* acc, double* W, cudaStream_t st) {
  using Ar = typename Arith<VS>::type;
  const int n = (int)A->n;
  const int rpw = 32 / r;
  const unsigned grid = grid_for_rows(n, r);
  const Ar a0 = Ar(1.0 / e), be0 = Ar(-c / e);
  const Ar a1 = Ar(2.0 / e), be1 = Ar(-2.0 * c / e);
  // step 0: Y_1 = Ahat V, acc = b0 V + b1 Y_1
  if (m == 1) {
    cheb_step_kernel<MS, VS, AccT, double, true><<<grid, kThreads, 0, st>>>(
        n, r, rpw, A->rowptr.p, A->col.p, val, v, nullptr, ya, nullptr, W, a0, be0, Ar(b[0]), Ar(b[1]));
    FLZ_LAUNCH_CHECK();
    return;
  }
  cheb_step_kernel<MS, VS, AccT, AccT, true><<<grid, kThreads, 0, st>>>(
      n, r, rpw, A->rowptr.p, A->col.p, val, v, nullptr, ya, nullptr, acc, a0, be0, Ar(b[0]), Ar(b[1]));
  FLZ_LAUNCH_CHECK();
  // Buffers: V is never written. Y_1 -> ya, Y_2 -> yb, then Y_{k+1}
  // overwrites Y_{k-1} in place.
  const VS* prev = v;
  const VS* cur = ya;
  for (int k = 1; k < m; ++k) {
    VS* next = (k == 1) ? yb : const_cast<VS*>(prev);
    if (k + 1 == m) {
      cheb_step_kernel<MS, VS, AccT, double, false><<<grid, kThreads, 0, st>>>(
          n, r, rpw, A->rowptr.p, A->col.p, val, cur, prev, next, acc, W, a1, be1, Ar(0), Ar(b[k + 1]));
    } else {
      cheb_step_kernel<MS, VS, AccT, AccT, false><<<grid, kThreads, 0, st>>>(
          n, r, rpw, A->rowptr.p, A->col.p, val, cur, prev, next, acc, acc, a1, be1, Ar(0), Ar(b[k + 1]));
    }
    FLZ_LAUNCH_CHECK();
    prev = cur;
    cur = next;
  }
}

// Y = A X, FP64, s columns (s <= 16), X and Y with row stride ld.
__global__ void __launch_bounds__(kThreads) spmm_kernel(int n, int s, int ld, int rows_per_warp,
                                                        const int* __restrict__ rowptr,
                                                        const int* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ X, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int sub = lane / s;
  const int c = lane - sub * s;
  const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const long long row = warp * rows_per_warp + sub;
  if (sub >= rows_per_warp || row >= n) return;
  double acc = 0.0;
  for (int j = __ldg(rowptr + row), je = __ldg(rowptr + row + 1); j < je; ++j)
    acc = fma(val[j], X[(size_t)__ldg(col + j) * ld + c], acc);
  Y[(size_t)row * ld + c] = acc;
}

}  // namespace

int filter_launch_count(int m, int precision) {
  if (m <= 0) return 1;
  return m + (precision == FLZ_PREC_FP64 ? 0 : 1);
}

void filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r, const double* V,
                  double* W, int precision, cudaStream_t st) {
  const size_t nr = (size_t)A->n * r;
  if (m == 0) {
    scale_kernel<<<grid_stride_blocks(nr), 256, 0, st>>>(V, W, coeffs[0], nr);
    FLZ_LAUNCH_CHECK();
    return;
  }
  if (precision == FLZ_PREC_FP64) {
    A->ws64.reserve(2 * nr);
    double* ya = A->ws64.p;
    double* yb = A->ws64.p + nr;
    // acc lives in W directly (FP64 output)
    run_recurrence<double, double, double>(A, A->val.p, c, e, coeffs, m, r, V, ya, yb, W, W, st);
  } else if (precision == FLZ_PREC_FP32) {
    if (!A->val32.p) {
      A->val32.reserve((size_t)A->nnz);
      convert_kernel<float><<<grid_stride_blocks(A->nnz), 256, 0, st>>>(A->val.p, A->val32.p, (size_t)A->nnz);
      FLZ_LAUNCH_CHECK();
    }
    A->ws32.reserve(4 * nr);
    float* vs = A->ws32.p;
    float* ya = vs + nr;
    float* yb = ya + nr;
    float* acc = yb + nr;
    convert_kernel<float><<<grid_stride_blocks(nr), 256, 0, st>>>(V, vs, nr);
    FLZ_LAUNCH_CHECK();
    run_recurrence<float, float, float>(A, A->val32.p, c, e, coeffs, m, r, vs, ya, yb, acc, W, st);
  } else if (precision == FLZ_PREC_BF16) {
    if (!A->val16.p) {
      A->val16.reserve((size_t)A->nnz);
      convert_kernel<__nv_bfloat16><<<grid_stride_blocks(A->nnz), 256, 0, st>>>(A->val.p, A->val16.p,
                                                                                (size_t)A->nnz);
      FLZ_LAUNCH_CHECK();
    }
    A->ws16.reserve(3 * nr);
    A->ws32.reserve(nr);
    __nv_bfloat16* vs = A->ws16.p;
    __nv_bfloat16* ya = vs + nr;
    __nv_bfloat16* yb = ya + nr;
    float* acc = A->ws32.p;
    convert_kernel<__nv_bfloat16><<<grid_stride_blocks(nr), 256, 0, st>>>(V, vs, nr);
    FLZ_LAUNCH_CHECK();
    run_recurrence<__nv_bfloat16, __nv_bfloat16, float>(A, A->val16.p, c, e, coeffs, m, r, vs, ya, yb, acc, W,
                                                        st);
  } else {
    fail(FLZ_ERR_INVALID_ARG, "unknown precision %d", precision);
  }
}

void spmm(const flz_matrix* A, const double* X, double* Y, int s, int ld, cudaStream_t st) {
  if (s < 1 || s > 16) fail(FLZ_ERR_INVALID_ARG, "spmm width %d out of range", s);
  spmm_kernel<<<grid_for_rows(A->n, s), kThreads, 0, st>>>((int)A->n, s, ld, 32 / s, A->rowptr.p, A->col.p,
                                                            A->val.p, X, Y);
  FLZ_LAUNCH_CHECK();
}

}  // namespace flz
