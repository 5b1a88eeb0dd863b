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
#include "device_common.cuh"
#include "flz_internal.h"

namespace flz {

using namespace dev;

namespace {

constexpr int kThreads = 256;

// One fused Chebyshev degree step over the whole matrix.
//   MS: storage of the scaled values 2 Ahat = (2/e)(A - cI) (the shift is
//       folded into the stored diagonal, the 2/e into every value), VS:
//       recurrence vector storage, AccS / OutS: running-sum input / output.
//   FIRST:  Y_1 = Ahat V = (1/2)(2 Ahat) V,      acc  = b_0 V + b_1 Y_1
//   else:   Y_{k+1} = (2 Ahat) Y_k - Y_{k-1},    acc += b_{k+1} Y_{k+1}
// The row sum starts from -Y_{k-1}, so a degree costs one multiply-add per
// stored entry and column plus one per element for the running sum.
// ynext may alias yprev; acc_out may alias acc_in (each element is read and
// written by the same thread).
template <class MS, class VS, class AccS, class OutS, bool FIRST>
__global__ void __launch_bounds__(kThreads) cheb_step_kernel(
    int n, int r, int rows_per_warp, const int* __restrict__ rowptr, const int* __restrict__ col,
    const MS* __restrict__ sval, const VS* __restrict__ ycur, const VS* yprev, VS* ynext, const AccS* acc_in,
    OutS* acc_out, typename Arith<VS>::type b_cur, typename Arith<VS>::type b_next) {
  using A = typename Arith<VS>::type;
  const int lane = threadIdx.x & 31;
  const int sub = lane / r;
  const int c = lane - sub * r;
  const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const long long row = warp * rows_per_warp + sub;
  if (sub >= rows_per_warp || row >= n) return;
  const size_t idx = (size_t)row * r + c;
  int j = __ldg(rowptr + row);
  const int jend = __ldg(rowptr + row + 1);
  A s = FIRST ? A(0) : -to_arith(yprev[idx]);
  for (; j + 4 <= jend; j += 4) {
    const int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2), c3 = __ldg(col + j + 3);
    const A a0 = to_arith(sval[j]), a1 = to_arith(sval[j + 1]), a2 = to_arith(sval[j + 2]), a3 = to_arith(sval[j + 3]);
    const A y0 = to_arith(ycur[(size_t)c0 * r + c]);
    const A y1 = to_arith(ycur[(size_t)c1 * r + c]);
    const A y2 = to_arith(ycur[(size_t)c2 * r + c]);
    const A y3 = to_arith(ycur[(size_t)c3 * r + c]);
    s = fma(a0, y0, s);
    s = fma(a1, y1, s);
    s = fma(a2, y2, s);
    s = fma(a3, y3, s);
  }
  for (; j < jend; ++j) s = fma(to_arith(sval[j]), to_arith(ycur[(size_t)__ldg(col + j) * r + c]), s);
  const A yn = FIRST ? A(0.5) * s : s;
  const VS yn_s = from_arith<VS>(yn);
  ynext[idx] = yn_s;
  const A yq = to_arith(yn_s);
  A acc = FIRST ? b_cur * to_arith(ycur[idx]) : A(to_arith(acc_in[idx]));
  acc = fma(b_next, yq, acc);
  acc_out[idx] = store_as<OutS>(acc);
}

constexpr int kRows = 256;  // rows per CTA in the row-per-thread kernel

// The fused degree step with one thread per row (all R columns) for R in
// {1, 2, 4, 8, 16}. The CTA's contiguous range of CSR indices and scaled
// values is first staged in shared memory with coalesced loads (when it fits
// `cap` entries; otherwise each thread reads its row from global memory), so
// the per-row reads that follow do not scatter across HBM sectors. A gathered
// row Y[col] is one R-wide vector load. Same arithmetic as cheb_step_kernel.
template <int R, class MS, class VS, class AccS, class OutS, bool FIRST>
__global__ void __launch_bounds__(kRows) cheb_rows_kernel(
    int n, int cap, int long_row, const int* __restrict__ rowptr, const int* __restrict__ col, const MS* __restrict__ sval,
    const VS* __restrict__ ycur, const VS* yprev, VS* ynext, const AccS* acc_in, OutS* acc_out,
    typename Arith<VS>::type b_cur, typename Arith<VS>::type b_next) {
  using A = typename Arith<VS>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  MS* s_val = reinterpret_cast<MS*>(smem);
  int* s_col = reinterpret_cast<int*>(smem + (size_t)cap * sizeof(MS));
  const int row0 = blockIdx.x * kRows;
  const int rend = min(n, row0 + kRows);
  const int row = row0 + (int)threadIdx.x;
  const int j0 = __ldg(rowptr + row0);
  const int j1 = __ldg(rowptr + rend);
  const bool staged = (j1 - j0) <= cap;  // uniform over the CTA
  if (staged) {
    for (int e = threadIdx.x; e < j1 - j0; e += kRows) {
      s_col[e] = __ldg(col + j0 + e);
      s_val[e] = sval[j0 + e];
    }
    __syncthreads();
  }
  allow_dependents();
  if (row >= n) return;
  const int jb = __ldg(rowptr + row);
  const int je = __ldg(rowptr + row + 1);
  if (je - jb > long_row) return;  // rows longer than long_row belong to cheb_long_kernel
  grid_dependency_wait();  // the vectors below are the previous degree's output
  A s[R];
  A acc[R];
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = A(0);
  } else {
    load_row<VS, R>(yprev + (size_t)row * R, s);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = -s[t];
    load_acc<R>(acc_in + (size_t)row * R, acc);  // issued early: it overlaps the gathers
  }
  // U independent row gathers in flight per thread (fewer for wide rows to
  // bound register use)
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
  store_row_rounded<VS, R>(ynext + (size_t)row * R, s);  // s now holds the stored (rounded) Y_next
  if (FIRST) {
    A v0[R];
    load_row<VS, R>(ycur + (size_t)row * R, v0);
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = b_cur * v0[t];
  }
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = fma(b_next, s[t], acc[t]);
  store_acc<R>(acc_out + (size_t)row * R, acc);
}

// The fused degree step on the SELL-32 layout (one warp per 32-row slice, one
// thread per row and all R columns): no shared-memory staging and no row
// pointers; a row's column indices and values are coalesced loads that do not
// depend on each other. Rows carrying the long-row marker are left to
// cheb_long_kernel. Same arithmetic as cheb_rows_kernel.
template <int R, class MS, class VS, class AccS, class OutS, bool FIRST>
__global__ void __launch_bounds__(kRows) cheb_sell_kernel(
    int n, const int* __restrict__ off, const int* __restrict__ scol, const MS* __restrict__ sval,
    const VS* __restrict__ ycur, const VS* yprev, VS* ynext, const AccS* acc_in, OutS* acc_out,
    typename Arith<VS>::type b_cur, typename Arith<VS>::type b_next) {
  using A = typename Arith<VS>::type;
  allow_dependents();
  const int row = blockIdx.x * kRows + (int)threadIdx.x;
  if (row >= n) return;
  const int sl = row >> 5;
  const int o = __ldg(off + sl);
  const int w = (__ldg(off + sl + 1) - o) >> 5;
  const int base = o + (row & 31);
  if (__ldg(scol + base) < 0) return;  // long row: cheb_long_kernel
  grid_dependency_wait();  // the vectors below are the previous degree's output
  A s[R];
  A acc[R];
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = A(0);
  } else {
    load_row<VS, R>(yprev + (size_t)row * R, s);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = -s[t];
    load_acc<R>(acc_in + (size_t)row * R, acc);
  }
  sell_row_sum<R, MS, VS, A>(scol, sval, base, w, ycur, s);
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] *= A(0.5);
  }
  store_row_rounded<VS, R>(ynext + (size_t)row * R, s);
  if (FIRST) {
    A v0[R];
    load_row<VS, R>(ycur + (size_t)row * R, v0);
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = b_cur * v0[t];
  }
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = fma(b_next, s[t], acc[t]);
  store_acc<R>(acc_out + (size_t)row * R, acc);
}

// The same degree step for rows with more than `long_row` stored entries
// (hubs of irregular graphs): one CTA per long row, its threads take strided
// entries and the partial sums are combined in shared memory, so a hub costs
// about (entries / 256) gathers of latency instead of `entries`.
template <int R, class MS, class VS, class AccS, class OutS, bool FIRST>
__global__ void __launch_bounds__(kRows) cheb_long_kernel(
    const int* __restrict__ long_rows, const int* __restrict__ rowptr, const int* __restrict__ col,
    const MS* __restrict__ sval, const VS* __restrict__ ycur, const VS* yprev, VS* ynext, const AccS* acc_in,
    OutS* acc_out, typename Arith<VS>::type b_cur, typename Arith<VS>::type b_next) {
  using A = typename Arith<VS>::type;
  __shared__ A red[kRows * R];
  const int row = long_rows[blockIdx.x];
  const int jb = __ldg(rowptr + row), je = __ldg(rowptr + row + 1);
  A s[R];
#pragma unroll
  for (int t = 0; t < R; ++t) s[t] = A(0);
  for (int j = jb + (int)threadIdx.x; j < je; j += kRows) {
    const A a = to_arith(sval[j]);
    A y[R];
    load_row<VS, R>(ycur + (size_t)__ldg(col + j) * R, y);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = fma(a, y[t], s[t]);
  }
#pragma unroll
  for (int t = 0; t < R; ++t) red[t * kRows + threadIdx.x] = s[t];
  __syncthreads();
  for (int h = kRows / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int t = 0; t < R; ++t) red[t * kRows + threadIdx.x] += red[t * kRows + threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  A yn[R], acc[R];
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < R; ++t) yn[t] = A(0.5) * red[t * kRows];
  } else {
    A yp[R];
    load_row<VS, R>(yprev + (size_t)row * R, yp);
#pragma unroll
    for (int t = 0; t < R; ++t) yn[t] = red[t * kRows] - yp[t];
    load_acc<R>(acc_in + (size_t)row * R, acc);
  }
  store_row_rounded<VS, R>(ynext + (size_t)row * R, yn);
  if (FIRST) {
    A v0[R];
    load_row<VS, R>(ycur + (size_t)row * R, v0);
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = b_cur * v0[t];
  }
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = fma(b_next, yn[t], acc[t]);
  store_acc<R>(acc_out + (size_t)row * R, acc);
}

template <class S>
__global__ void convert_kernel(const double* __restrict__ in, S* __restrict__ out, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = from_arith<S>((typename Arith<S>::type)in[i]);
}

template <class T>
__global__ void scale_kernel(const T* __restrict__ in, T* __restrict__ out, T s, size_t count) {
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

template <class MS, class VS, class AccT, class WT>
void run_lanes(const flz_matrix* A, const MS* val, const double* b, int m, int r, const VS* v, VS* ya, VS* yb,
               AccT* acc, WT* W, cudaStream_t st) {
  using Ar = typename Arith<VS>::type;
  const int n = (int)A->n;
  const int rpw = 32 / r;
  const unsigned grid = grid_for_rows(n, r);
  // step 0: Y_1 = Ahat V, acc = b0 V + b1 Y_1
  if (m == 1) {
    cheb_step_kernel<MS, VS, AccT, WT, true><<<grid, kThreads, 0, st>>>(
        n, r, rpw, A->rowptr.p, A->col.p, val, v, nullptr, ya, nullptr, W, Ar(b[0]), Ar(b[1]));
    FLZ_LAUNCH_CHECK();
    return;
  }
  cheb_step_kernel<MS, VS, AccT, AccT, true><<<grid, kThreads, 0, st>>>(
      n, r, rpw, A->rowptr.p, A->col.p, val, v, nullptr, ya, nullptr, acc, Ar(b[0]), Ar(b[1]));
  FLZ_LAUNCH_CHECK();
  // Buffers: V is never written. Y_1 -> ya, Y_2 -> yb, then Y_{k+1}
  // overwrites Y_{k-1} in place.
  const VS* prev = v;
  const VS* cur = ya;
  for (int k = 1; k < m; ++k) {
    VS* next = (k == 1) ? yb : const_cast<VS*>(prev);
    if (k + 1 == m) {
      cheb_step_kernel<MS, VS, AccT, WT, false><<<grid, kThreads, 0, st>>>(
          n, r, rpw, A->rowptr.p, A->col.p, val, cur, prev, next, acc, W, Ar(0), Ar(b[k + 1]));
    } else {
      cheb_step_kernel<MS, VS, AccT, AccT, false><<<grid, kThreads, 0, st>>>(
          n, r, rpw, A->rowptr.p, A->col.p, val, cur, prev, next, acc, acc, Ar(0), Ar(b[k + 1]));
    }
    FLZ_LAUNCH_CHECK();
    prev = cur;
    cur = next;
  }
}

template <int R, class MS, class VS, class AccT, class WT>
void run_rows(const flz_matrix* A, const MS* val, const double* b, int m, const VS* v, VS* ya, VS* yb, AccT* acc,
              WT* W, cudaStream_t st) {
  using Ar = typename Arith<VS>::type;
  const int n = (int)A->n;
  const int cap = std::min<int>(A->max_cta_nnz, 4096);
  const size_t smem = (size_t)cap * (sizeof(MS) + sizeof(int));
  const unsigned grid = (unsigned)((n + kRows - 1) / kRows);
  const int* rp = A->rowptr.p;
  const int* cl = A->col.p;
  const int nl = A->n_long;
  const int thr = nl > 0 ? kLongRow : 0x7fffffff;
  const int* lr = A->long_rows.p;
  auto step = [&](bool first, bool last, const VS* cur, const VS* prev, VS* next, Ar bc, Ar bn) {
    if (first && last) {
      cheb_rows_kernel<R, MS, VS, AccT, WT, true><<<grid, kRows, smem, st>>>(n, cap, thr, rp, cl, val, cur, prev, next, acc, W, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, WT, true><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, W, bc, bn);
    } else if (first) {
      cheb_rows_kernel<R, MS, VS, AccT, AccT, true><<<grid, kRows, smem, st>>>(n, cap, thr, rp, cl, val, cur, prev, next, acc, acc, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, AccT, true><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, acc, bc, bn);
    } else if (last) {
      // degree steps after the first overlap their CSR staging with the
      // previous step's tail (programmatic dependent launch)
      launch_dependent(cheb_rows_kernel<R, MS, VS, AccT, WT, false>, grid, kRows, smem, st, n, cap, thr, rp, cl, val,
                       cur, prev, next, acc, W, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, WT, false><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, W, bc, bn);
    } else {
      launch_dependent(cheb_rows_kernel<R, MS, VS, AccT, AccT, false>, grid, kRows, smem, st, n, cap, thr, rp, cl,
                       val, cur, prev, next, acc, acc, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, AccT, false><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, acc, bc, bn);
    }
    if (nl) FLZ_LAUNCH_CHECK();
  };
  // step 0 reads V, writes Y_1 to ya; then Y_{k+1} overwrites Y_{k-1} in place
  step(true, m == 1, v, nullptr, ya, Ar(b[0]), Ar(b[1]));
  const VS* prev = v;
  const VS* cur = ya;
  for (int k = 1; k < m; ++k) {
    VS* next = (k == 1) ? yb : const_cast<VS*>(prev);
    step(false, k + 1 == m, cur, prev, next, Ar(0), Ar(b[k + 1]));
    prev = cur;
    cur = next;
  }
}

template <int R, class MS, class VS, class AccT, class WT>
void run_sell(const flz_matrix* A, const MS* vsell, const MS* val, const double* b, int m, const VS* v, VS* ya,
              VS* yb, AccT* acc, WT* W, cudaStream_t st) {
  using Ar = typename Arith<VS>::type;
  const int n = (int)A->n;
  const unsigned grid = (unsigned)((n + kRows - 1) / kRows);
  const int* of = A->sell_off.p;
  const int* sc = A->sell_col.p;
  const int* rp = A->rowptr.p;
  const int* cl = A->col.p;
  const int nl = A->n_long;
  const int* lr = A->long_rows.p;
  auto step = [&](bool first, bool last, const VS* cur, const VS* prev, VS* next, Ar bc, Ar bn) {
    if (first && last) {
      cheb_sell_kernel<R, MS, VS, AccT, WT, true><<<grid, kRows, 0, st>>>(n, of, sc, vsell, cur, prev, next, acc, W, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, WT, true><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, W, bc, bn);
    } else if (first) {
      cheb_sell_kernel<R, MS, VS, AccT, AccT, true><<<grid, kRows, 0, st>>>(n, of, sc, vsell, cur, prev, next, acc, acc, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, AccT, true><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, acc, bc, bn);
    } else if (last) {
      launch_dependent(cheb_sell_kernel<R, MS, VS, AccT, WT, false>, grid, kRows, 0, st, n, of, sc, vsell, cur, prev,
                       next, acc, W, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, WT, false><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, W, bc, bn);
    } else {
      launch_dependent(cheb_sell_kernel<R, MS, VS, AccT, AccT, false>, grid, kRows, 0, st, n, of, sc, vsell, cur,
                       prev, next, acc, acc, bc, bn);
      FLZ_LAUNCH_CHECK();
      if (nl) cheb_long_kernel<R, MS, VS, AccT, AccT, false><<<nl, kRows, 0, st>>>(lr, rp, cl, val, cur, prev, next, acc, acc, bc, bn);
    }
    if (nl) FLZ_LAUNCH_CHECK();
  };
  step(true, m == 1, v, nullptr, ya, Ar(b[0]), Ar(b[1]));
  const VS* prev = v;
  const VS* cur = ya;
  for (int k = 1; k < m; ++k) {
    VS* next = (k == 1) ? yb : const_cast<VS*>(prev);
    step(false, k + 1 == m, cur, prev, next, Ar(0), Ar(b[k + 1]));
    prev = cur;
    cur = next;
  }
}

inline bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Row-per-thread kernel for r in {1, 2, 4, 8, 16} when every block is aligned
// for R-wide vector access; the lane-per-column kernel otherwise.
template <class MS, class VS, class AccT, class WT>
void run_recurrence(const flz_matrix* A, const MS* vsell, const MS* val, const double* b, int m, int r, const VS* v,
                    VS* ya, VS* yb, AccT* acc, WT* W, cudaStream_t st) {
  if (vsell) {  // SELL-32 layout (the caller checked width and alignment)
    switch (r) {
      case 1: run_sell<1, MS, VS, AccT, WT>(A, vsell, val, b, m, v, ya, yb, acc, W, st); break;
      case 2: run_sell<2, MS, VS, AccT, WT>(A, vsell, val, b, m, v, ya, yb, acc, W, st); break;
      case 3: run_sell<3, MS, VS, AccT, WT>(A, vsell, val, b, m, v, ya, yb, acc, W, st); break;
      case 4: run_sell<4, MS, VS, AccT, WT>(A, vsell, val, b, m, v, ya, yb, acc, W, st); break;
      case 8: run_sell<8, MS, VS, AccT, WT>(A, vsell, val, b, m, v, ya, yb, acc, W, st); break;
      default: run_sell<16, MS, VS, AccT, WT>(A, vsell, val, b, m, v, ya, yb, acc, W, st); break;
    }
    return;
  }
  // the staged-CSR row kernel serves power-of-two widths; r = 3 runs row per
  // thread only in the SELL-32 layout (else the lane-per-column kernel)
  const bool pow2 = row_kernel_width(r) && r != 3;
  const size_t av = row_alignment(r, sizeof(VS));
  const size_t aa = row_alignment(r, sizeof(AccT));
  const size_t aw = row_alignment(r, sizeof(WT));
  const bool ok = pow2 && A->max_cta_nnz > 0 && aligned_to(v, av) && aligned_to(ya, av) && aligned_to(yb, av) &&
                  aligned_to(acc, aa) && aligned_to(W, aw);
  if (!ok) {
    run_lanes<MS, VS, AccT, WT>(A, val, b, m, r, v, ya, yb, acc, W, st);
    return;
  }
  switch (r) {
    case 1: run_rows<1, MS, VS, AccT, WT>(A, val, b, m, v, ya, yb, acc, W, st); break;
    case 2: run_rows<2, MS, VS, AccT, WT>(A, val, b, m, v, ya, yb, acc, W, st); break;
    case 4: run_rows<4, MS, VS, AccT, WT>(A, val, b, m, v, ya, yb, acc, W, st); break;
    case 8: run_rows<8, MS, VS, AccT, WT>(A, val, b, m, v, ya, yb, acc, W, st); break;
    default: run_rows<16, MS, VS, AccT, WT>(A, val, b, m, v, ya, yb, acc, W, st); break;
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

// 2 Ahat in storage precision `prec`, rebuilt only when (c, e) change.
template <class S>
const S* scaled(flz_matrix* A, DevBuf<S>& buf, int prec, double c, double e, cudaStream_t st) {
  if (!(A->sc_ok[prec] && A->sc_c[prec] == c && A->sc_e[prec] == e && buf.p)) {
    buf.reserve((size_t)A->nnz);
    scale_values<S>(A, c, e, buf.p, st);
    A->sc_c[prec] = c;
    A->sc_e[prec] = e;
    A->sc_ok[prec] = true;
  }
  return buf.p;
}

// The same in the SELL-32 layout.
template <class S>
const S* scaled_sell(flz_matrix* A, DevBuf<S>& buf, int prec, double c, double e, cudaStream_t st) {
  if (!(A->ss_ok[prec] && A->ss_c[prec] == c && A->ss_e[prec] == e && buf.p)) {
    buf.reserve((size_t)A->sell_len);
    scale_values_sell<S>(A, c, e, buf.p, st);
    A->ss_c[prec] = c;
    A->ss_e[prec] = e;
    A->ss_ok[prec] = true;
  }
  return buf.p;
}

// The filter's view of 2 Ahat: the SELL-32 values when that kernel runs
// (power-of-two r, aligned blocks, a matrix with little padding), the CSR
// values for the other kernels (and for long rows next to SELL).
template <class S>
struct ScaledMatrix {
  const S* sell = nullptr;
  const S* csr = nullptr;
};

template <class S>
ScaledMatrix<S> prepare(flz_matrix* A, DevBuf<S>& csr_buf, DevBuf<S>& sell_buf, int prec, double c, double e,
                        bool use_sell, cudaStream_t st) {
  ScaledMatrix<S> out;
  if (use_sell) out.sell = scaled_sell<S>(A, sell_buf, prec, c, e, st);
  if (!use_sell || A->n_long > 0) out.csr = scaled<S>(A, csr_buf, prec, c, e, st);
  return out;
}

// SELL-32 needs the row-per-thread form: r in {1, 2, 3, 4, 8, 16} and aligned
// access to the caller's blocks (the library's own scratch is always aligned).
// The FP64 step is bound by the FP64 pipe, where every padding entry costs a
// multiply-add like a stored one: FP64 takes SELL-32 only when the padding is
// at most 10 % of the stored entries (the memory-bound precisions up to the
// layout's own 30 %).
bool sell_usable(const flz_matrix* A, int r, const void* v, size_t v_elem, const void* w, size_t w_elem,
                 bool fp64 = false) {
  if (fp64 && (double)A->sell_len > 1.10 * (double)A->nnz) return false;
  return A->sell && row_kernel_width(r) && aligned_to(v, row_alignment(r, v_elem)) &&
         aligned_to(w, row_alignment(r, w_elem));
}

}  // namespace

void filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r, const double* V,
                  double* W, int precision, int recurrence, cudaStream_t st) {
  const size_t nr = (size_t)A->n * r;
  if (m == 0) {
    scale_kernel<double><<<grid_stride_blocks(nr), 256, 0, st>>>(V, W, coeffs[0], nr);
    FLZ_LAUNCH_CHECK();
    return;
  }
  const bool clen = recurrence == FLZ_REC_CLENSHAW;
  if (precision == FLZ_PREC_FX64) {
    if (clen) fail(FLZ_ERR_INVALID_ARG, "the fixed-point filter evaluates the forward recurrence only");
    if (fx_filter_apply(A, c, e, coeffs, m, r, V, W, st)) {
      A->last_filter_precision = FLZ_PREC_FX64;
      return;
    }
    precision = FLZ_PREC_FP64;  // the format does not apply to this matrix or block: FP64 arithmetic
  }
  A->last_filter_precision = precision;
  if (precision == FLZ_PREC_FP64) {
    const auto M = prepare<double>(A, A->sval64, A->ssell64, 0, c, e, sell_usable(A, r, V, 8, W, 8, true), st);
    A->ws64.reserve(2 * nr);
    double* ya = A->ws64.p;
    double* yb = A->ws64.p + nr;
    if (clen)
      run_clenshaw<double, double, double>(A, M.sell, M.csr, coeffs, m, r, V, ya, yb, W, st);
    else  // the running sum lives in W directly (FP64 output)
      run_recurrence<double, double, double, double>(A, M.sell, M.csr, coeffs, m, r, V, ya, yb, W, W, st);
  } else if (precision == FLZ_PREC_FP32) {
    A->ws32.reserve(4 * nr);
    float* vs = A->ws32.p;
    float* ya = vs + nr;
    float* yb = ya + nr;
    float* acc = yb + nr;
    const auto M = prepare<float>(A, A->sval32, A->ssell32, 1, c, e, sell_usable(A, r, vs, 4, W, 8), st);
    convert_kernel<float><<<grid_stride_blocks(nr), 256, 0, st>>>(V, vs, nr);
    FLZ_LAUNCH_CHECK();
    if (clen)
      run_clenshaw<float, float, double>(A, M.sell, M.csr, coeffs, m, r, vs, ya, yb, W, st);
    else
      run_recurrence<float, float, float, double>(A, M.sell, M.csr, coeffs, m, r, vs, ya, yb, acc, W, st);
  } else if (precision == FLZ_PREC_BF16) {
    A->ws16.reserve(3 * nr);
    __nv_bfloat16* vs = A->ws16.p;
    __nv_bfloat16* ya = vs + nr;
    __nv_bfloat16* yb = ya + nr;
    const auto M = prepare<__nv_bfloat16>(A, A->sval16, A->ssell16, 2, c, e, sell_usable(A, r, vs, 2, W, 8), st);
    convert_kernel<__nv_bfloat16><<<grid_stride_blocks(nr), 256, 0, st>>>(V, vs, nr);
    FLZ_LAUNCH_CHECK();
    if (clen) {
      run_clenshaw<__nv_bfloat16, __nv_bfloat16, double>(A, M.sell, M.csr, coeffs, m, r, vs, ya, yb, W, st);
    } else {
      A->ws32.reserve(nr);
      float* acc = A->ws32.p;
      run_recurrence<__nv_bfloat16, __nv_bfloat16, float, double>(A, M.sell, M.csr, coeffs, m, r, vs, ya, yb, acc, W,
                                                                  st);
    }
  } else if (precision == FLZ_PREC_DF64) {
    A->wsdf.reserve(4 * nr);
    dfloat* vs = A->wsdf.p;
    dfloat* ya = vs + nr;
    dfloat* yb = ya + nr;
    dfloat* acc = yb + nr;
    const auto M = prepare<dfloat>(A, A->svaldf, A->sselldf, 3, c, e, sell_usable(A, r, vs, 8, W, 8), st);
    convert_kernel<dfloat><<<grid_stride_blocks(nr), 256, 0, st>>>(V, vs, nr);
    FLZ_LAUNCH_CHECK();
    if (clen)
      run_clenshaw<dfloat, dfloat, double>(A, M.sell, M.csr, coeffs, m, r, vs, ya, yb, W, st);
    else
      run_recurrence<dfloat, dfloat, dfloat, double>(A, M.sell, M.csr, coeffs, m, r, vs, ya, yb, acc, W, st);
  } else {
    fail(FLZ_ERR_INVALID_ARG, "unknown precision %d", precision);
  }
}

void filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r, const dfloat* V,
                  dfloat* W, int recurrence, cudaStream_t st) {
  const size_t nr = (size_t)A->n * r;
  if (m == 0) {
    scale_kernel<dfloat><<<grid_stride_blocks(nr), 256, 0, st>>>(V, W, dfloat(coeffs[0]), nr);
    FLZ_LAUNCH_CHECK();
    return;
  }
  const auto M = prepare<dfloat>(A, A->svaldf, A->sselldf, 3, c, e, sell_usable(A, r, V, 8, W, 8), st);
  A->wsdf.reserve(2 * nr);
  dfloat* ya = A->wsdf.p;
  dfloat* yb = ya + nr;
  if (recurrence == FLZ_REC_CLENSHAW)
    run_clenshaw<dfloat, dfloat, dfloat>(A, M.sell, M.csr, coeffs, m, r, V, ya, yb, W, st);
  else  // the running sum lives in W directly
    run_recurrence<dfloat, dfloat, dfloat, dfloat>(A, M.sell, M.csr, coeffs, m, r, V, ya, yb, W, W, st);
}

void spmm(const flz_matrix* A, const double* X, double* Y, int s, int ld, cudaStream_t st) {
  if (s < 1 || s > 16) fail(FLZ_ERR_INVALID_ARG, "spmm width %d out of range", s);
  spmm_kernel<<<grid_for_rows(A->n, s), kThreads, 0, st>>>((int)A->n, s, ld, 32 / s, A->rowptr.p, A->col.p,
                                                            A->val.p, X, Y);
  FLZ_LAUNCH_CHECK();
}

}  // namespace flz
