// W = p_m(Ahat) V (Section 2.2, forward recurrence eq. def:cheb1 with the
// running sum fused) in 64-bit fixed point on the integer pipes.
//
// Why: on this GPU FP64 runs at a small fraction of the FP32 and integer
// rates, and the FP64 degree step is bound by the FP64 pipe, not by HBM. The
// recurrence's values are bounded, which fixed point needs: with the spectrum
// of Ahat in [-1, 1] and a column v of V, every entry of T_k(Ahat) v is at
// most ||v||_2 in magnitude, and the entries of 2 Ahat are at most 2.
//
// Number format.
//   vectors Y_k, running sum:  integers in units of 2^-F of the column's
//                              scale 2^E (2^E about ||v||_2), |Y| < 2^(63-F);
//                              F = 61 when every row of 2 Ahat has absolute
//                              sum at most 2.1 (stencils), else F = 60
//   2 Ahat, coefficients b_k:  integers in units of 2^-61, |.| < 4
// Both are stored offset-binary (u = x + 2^63, the sign bit flipped), so all
// 32-bit limb products are unsigned. A row sum
//   sum_j a_j y_j = sum_j a'_j y'_j - 2^63 (sum_j a'_j + sum_j y'_j) + cnt 2^126
// is accumulated in its top 96 bits (the low 32 bits of a'_0 y'_0 are left
// out: less than 2^-28 of the result's unit in all) with carry chains, then
// shifted and rounded once to the result's units: one rounding per row,
// column and degree, at 2^-(F+1) of the column scale (FP64 rounds each
// partial sum at 2^-53 of its magnitude). Everything wraps modulo 2^64 and
// the result is exact as long as it fits, which the overflow check
// guarantees: a new value above 1.25 in magnitude (the spectrum outside
// [-1, 1]) raises a flag instead of wrapping (it cannot wrap first: with row
// sums of |2 Ahat| at most L, a step starting below 1.25 ends below
// 1.25 (L + 1) < 2^(63-F), the bound F is chosen by).
//
// Per stored entry and column: 9 integer multiply-adds and two adds on the
// integer pipes; no FP64 arithmetic in the degree steps.
#include <cmath>
#include <cstring>

#include "flz_internal.h"
#include "tcgen05.cuh"

namespace flz {

using namespace dev;

namespace {

constexpr uint64_t kOff = 0x8000000000000000ull;  // offset of the offset-binary form
constexpr int kValBits = 61;                        // fractional bits of 2 Ahat and b_k
constexpr int kThreads = 256;

// Top 96 bits (w1 w2 w3 at 2^32, 2^64, 2^96) of a sum of 64 x 64-bit unsigned
// products, and the sum of the y operands.
struct Acc {
  uint32_t w1, w2, w3;
  uint64_t sy;
};

__device__ __forceinline__ void acc_init(Acc& s, int shift) {
  s.w1 = 1u << (shift - 33);  // + 2^(shift-1): round to nearest on the final shift
  s.w2 = 0u;
  s.w3 = 0u;
  s.sy = 0ull;
}

// s += a * y (a, y offset-binary operands), exact in the top 96 bits
__device__ __forceinline__ void mac(Acc& s, uint64_t a, uint64_t y) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
  asm("mad.hi.cc.u32  %0, %3, %4, %0;\n\t"   // w1 += hi(a0 y0)
      "madc.lo.cc.u32 %1, %5, %6, %1;\n\t"   // w2 += lo(a1 y1) + c
      "madc.hi.u32    %2, %5, %6, %2;\n\t"   // w3 += hi(a1 y1) + c
      "mad.lo.cc.u32  %0, %3, %6, %0;\n\t"   // w1 += lo(a0 y1)
      "madc.hi.cc.u32 %1, %3, %6, %1;\n\t"   // w2 += hi(a0 y1) + c
      "addc.u32       %2, %2, 0;\n\t"
      "mad.lo.cc.u32  %0, %5, %4, %0;\n\t"   // w1 += lo(a1 y0)
      "madc.hi.cc.u32 %1, %5, %4, %1;\n\t"   // w2 += hi(a1 y0) + c
      "addc.u32       %2, %2, 0;"
      : "+r"(s.w1), "+r"(s.w2), "+r"(s.w3)
      : "r"(a0), "r"(y0), "r"(a1), "r"(y1));
  s.sy += y;
}

// s += t (a partial sum of another thread)
__device__ __forceinline__ void acc_add(Acc& s, const Acc& t) {
  asm("add.cc.u32  %0, %0, %3;\n\t"
      "addc.cc.u32 %1, %1, %4;\n\t"
      "addc.u32    %2, %2, %5;"
      : "+r"(s.w1), "+r"(s.w2), "+r"(s.w3)
      : "r"(t.w1), "r"(t.w2), "r"(t.w3));
  s.sy += t.sy;
}

// round(sum a y / 2^shift) modulo 2^64 for shift 61 or 62, given sa = sum a'
__device__ __forceinline__ uint64_t acc_result(const Acc& s, uint64_t sa, int shift) {
  const uint64_t lo = (((uint64_t)s.w2 << 32) | s.w1) >> (shift - 32);
  const uint64_t hi = (uint64_t)s.w3 << (96 - shift);
  return (lo | hi) - ((sa + s.sy) << (63 - shift));
}

// round(b y) in units of 2^-60 for the offset-binary coefficient bo and value yo
__device__ __forceinline__ uint64_t coeff_times(uint64_t bo, uint64_t yo) {
  Acc s;
  acc_init(s, kValBits);
  mac(s, bo, yo);
  return acc_result(s, bo, kValBits);
}

// flags |Y| >= 1.25 in column-scale units (limit = 1.25 2^F)
__device__ __forceinline__ void check_range(uint64_t yo, uint64_t limit, unsigned* flag) {
  if (yo - (kOff - limit) >= 2 * limit) atomicOr(flag, 1u);
}

__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// Per-degree parameters of the fixed-point step.
struct FxStep {
  uint64_t b_cur;    // b_0 (first step only), offset-binary, units 2^-61 scaled by 2^-s
  uint64_t b_next;   // b_{k+1}
  uint64_t b_m1;     // b_k     (batches: the terms added three at a time)
  uint64_t b_m2;     // b_{k-1}
  int t;             // k + 1: the index of the value this step forms
  const int* cexp;   // column scale exponents E_t
  int sum_exp;       // s: the running sum is held in units of 2^(s - F)
  int vec_bits;      // F
  uint64_t limit;    // 1.25 2^F: larger values are flagged
  unsigned* flag;    // bit 0: a value left the range; bit 1: a stage wait expired
  uint64_t wait_ns;  // limit of each barrier wait
};

template <int R>
__device__ __forceinline__ void load_u64_row(const uint64_t* p, uint64_t (&v)[R]) {
  if constexpr ((R & 1) == 0) {
#pragma unroll
    for (int i = 0; i < R; i += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p + i);
      v[i] = t.x;
      v[i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = p[i];
  }
}
// The same through L2 only (__ldcg): values another CTA of the same launch
// wrote (the persistent batch kernel), never a stale L1 line.
template <int R>
__device__ __forceinline__ void load_u64_row_cg(const uint64_t* p, uint64_t (&v)[R]) {
  if constexpr ((R & 1) == 0) {
#pragma unroll
    for (int i = 0; i < R; i += 2) {
      const ulonglong2 t = __ldcg(reinterpret_cast<const ulonglong2*>(p + i));
      v[i] = t.x;
      v[i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = __ldcg(reinterpret_cast<const unsigned long long*>(p + i));
  }
}

template <int R, class T>
__device__ __forceinline__ void store_u64_row(T* p, const T (&v)[R]) {
  if constexpr ((R & 1) == 0) {
#pragma unroll
    for (int i = 0; i < R; i += 2) {
      if constexpr (std::is_same<T, double>::value)
        *reinterpret_cast<double2*>(p + i) = make_double2(v[i], v[i + 1]);
      else
        *reinterpret_cast<ulonglong2*>(p + i) = make_ulonglong2((unsigned long long)v[i], (unsigned long long)v[i + 1]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) p[i] = v[i];
  }
}

// The end of a row's degree step, shared by the kernels: from the row sums
// to Y_{k+1}, the running sum and (last step) W. own: the row's V (first
// step) or Y_{k-1}; sum: its running sum (not read in the first step).
template <int R, bool FIRST, bool LAST>
__device__ __forceinline__ void finish_row(size_t idx, const Acc (&S)[R], uint64_t sa, const uint64_t (&own)[R],
                                           uint64_t (&sum)[R], uint64_t* ynext, uint64_t* acc, double* W,
                                           const FxStep& k) {
  uint64_t yn[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    if (FIRST) {
      yn[t] = acc_result(S[t], sa, kValBits + 1) + kOff;  // Y_1 = (1/2)(2 Ahat) V
      sum[t] = coeff_times(k.b_cur, own[t]) + coeff_times(k.b_next, yn[t]);
    } else {
      yn[t] = acc_result(S[t], sa, kValBits) - own[t];  // Y_{k+1} = 2 Ahat Y_k - Y_{k-1}
      sum[t] += coeff_times(k.b_next, yn[t]);
    }
    check_range(yn[t], k.limit, k.flag);
  }
  if (!LAST) {
    store_u64_row<R>(ynext + idx, yn);
    store_u64_row<R>(acc + idx, sum);
  } else {
    double w[R];
#pragma unroll
    for (int t = 0; t < R; ++t)
      w[t] = __ll2double_rn((long long)sum[t]) * pow2(k.cexp[t] + k.sum_exp - k.vec_bits);
    store_u64_row<R>(W + idx, w);
  }
}

// finish_row with the row's own values read from global memory
template <int R, bool FIRST, bool LAST>
__device__ __forceinline__ void finish_row_global(size_t idx, const Acc (&S)[R], uint64_t sa, const uint64_t* ycur,
                                                  const uint64_t* yprev, uint64_t* ynext, uint64_t* acc, double* W,
                                                  const FxStep& k) {
  uint64_t own[R], sum[R];
  load_u64_row<R>((FIRST ? ycur : yprev) + idx, own);
  if (!FIRST) load_u64_row<R>(acc + idx, sum);
  finish_row<R, FIRST, LAST>(idx, S, sa, own, sum, ynext, acc, W, k);
}

// Batches read and write the running sum sum_k b_k Y_k every third degree
// only: the step forming Y_t (t = k + 1) also holds Y_{k-1} (its recurrence
// operand) and reads its own row of Y_k, so it adds the terms of indices
// t-2, t-1, t when t = 1 (mod 3), and the pending one or two at the last
// step. Each term is rounded once and the sums are exact integers, so the
// result is the same as adding every term at its own step. (The single
// problem's staged kernel is faster with a term per step: there the saved
// bytes do not pay for the registers the extra terms take.)
__device__ __forceinline__ int flush_terms(int t, bool last) {
  const int p = (t - 1) % 3;
  return p == 0 ? 3 : (last ? p : 0);
}

// finish_row with the terms added three at a time; sum is read only when
// terms are added, ycur (Y_k) only when two or more are.
template <int R, bool FIRST, bool LAST, bool CG = false>
__device__ __forceinline__ void finish_row_flush3(size_t idx, const Acc (&S)[R], uint64_t sa,
                                                  const uint64_t (&own)[R], uint64_t (&sum)[R],
                                                  const uint64_t* ycur, uint64_t* ynext, uint64_t* acc, double* W,
                                                  const FxStep& k) {
  const int nt = FIRST ? 2 : flush_terms(k.t, LAST);
  uint64_t yk[R];
  if (!FIRST && nt >= 2) {
    if (CG) load_u64_row_cg<R>(ycur + idx, yk);
    else load_u64_row<R>(ycur + idx, yk);
  }
  uint64_t yn[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    if (FIRST) {
      yn[t] = acc_result(S[t], sa, kValBits + 1) + kOff;  // Y_1 = (1/2)(2 Ahat) V
      sum[t] = coeff_times(k.b_cur, own[t]) + coeff_times(k.b_next, yn[t]);
    } else {
      yn[t] = acc_result(S[t], sa, kValBits) - own[t];  // Y_{k+1} = 2 Ahat Y_k - Y_{k-1}
      if (nt >= 1) sum[t] += coeff_times(k.b_next, yn[t]);
      if (nt >= 2) sum[t] += coeff_times(k.b_m1, yk[t]);
      if (nt >= 3) sum[t] += coeff_times(k.b_m2, own[t]);
    }
    check_range(yn[t], k.limit, k.flag);
  }
  if (!LAST) {
    store_u64_row<R>(ynext + idx, yn);
    if (nt > 0) store_u64_row<R>(acc + idx, sum);
  } else {
    double w[R];
#pragma unroll
    for (int t = 0; t < R; ++t)
      w[t] = __ll2double_rn((long long)sum[t]) * pow2(k.cexp[t] + k.sum_exp - k.vec_bits);
    store_u64_row<R>(W + idx, w);
  }
}

// Bounded wait for phase 0 of a CTA barrier: false after wait_ns (2 s unless
// flz_set_wait_limit changed it), with bit 1 of the flag word set (reported as
// a timeout).
__device__ __forceinline__ bool stage_wait(uint64_t* bar, unsigned* flag, uint64_t wait_ns) {
  if (wait_ns == 0) {  // a zero limit: one non-blocking test, no waiting at all
    if (tc::mbar_test_wait(bar, 0)) return true;
    atomicOr(flag, 2u);
    return false;
  }
  if (tc::mbar_try_wait(bar, 0)) return true;
  const uint64_t t0 = tc::globaltimer();
  while (!tc::mbar_try_wait(bar, 0))
    if (tc::globaltimer() - t0 > wait_ns) {
      atomicOr(flag, 2u);
      return false;
    }
  return true;
}

// The fused degree step on the SELL-32 layout, one thread per row and all R
// columns (entry j of a row at base + 32 j), staged through shared memory:
// a CTA's 256 rows are 8 slices whose column indices and values form one
// contiguous range, fetched by bulk (TMA) copies BEFORE the wait on the
// previous degree (they are constant), so the matrix stream overlaps that
// degree's tail; after the wait, the CTA's rows of Y_{k-1} (V in the first
// step) and of the running sum arrive the same way while the threads gather
// Y_k. Each row's chain of dependent memory round trips shrinks to the
// gathers. Rows of a CTA whose vector rows do not form a 16-byte multiple
// (odd tails), or a W not 16-byte aligned (vec_bulk = 0), read them directly.
// ynext may alias yprev; W (last step) may alias acc.
template <int R, int U, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads) fx_sell_kernel(int n, int nsl, int emax, int vec_bulk,
                                                           const int* __restrict__ off, const int* __restrict__ scol,
                                                           const uint64_t* __restrict__ sval,
                                                           const uint64_t* __restrict__ ycur, const uint64_t* yprev,
                                                           uint64_t* ynext, uint64_t* acc, double* W, FxStep k) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);         // [0] matrix range, [1] vector rows
  uint64_t* s_own = reinterpret_cast<uint64_t*>(smem + 16);  // V (first step) or Y_{k-1} rows
  uint64_t* s_sum = s_own + kThreads * R;                    // running-sum rows
  uint64_t* s_val = s_sum + kThreads * R;
  int* s_col = reinterpret_cast<int*>(s_val + emax);
  const int sl0 = blockIdx.x * 8, sl1 = min(nsl, sl0 + 8);
  const int e0 = __ldg(off + sl0), e1 = __ldg(off + sl1);
  const int row0 = blockIdx.x * kThreads, rows = min(kThreads, n - row0);
  const bool vb = vec_bulk && ((rows * R) % 2 == 0);  // uniform over the CTA
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
    tc::mbar_expect_tx(&bar[0], (uint32_t)(e1 - e0) * 12u);
    tc::bulk_g2s(s_val, sval + e0, (uint32_t)(e1 - e0) * 8u, &bar[0]);
    tc::bulk_g2s(s_col, scol + e0, (uint32_t)(e1 - e0) * 4u, &bar[0]);
  }
  __syncthreads();
  allow_dependents();
  grid_dependency_wait();  // the vectors below are the previous degree's output
  if (threadIdx.x == 0 && vb) {
    const uint32_t bytes = (uint32_t)rows * R * 8u;
    const size_t at = (size_t)row0 * R;
    if (FIRST) {
      tc::mbar_expect_tx(&bar[1], bytes);
      tc::bulk_g2s(s_own, ycur + at, bytes, &bar[1]);
    } else {
      tc::mbar_expect_tx(&bar[1], 2 * bytes);
      tc::bulk_g2s(s_own, yprev + at, bytes, &bar[1]);
      tc::bulk_g2s(s_sum, acc + at, bytes, &bar[1]);
    }
  }
  const int t = threadIdx.x, row = row0 + t;
  Acc S[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc_init(S[c], FIRST ? kValBits + 1 : kValBits);
  uint64_t sa = 0;
  bool active = row < n;
  const bool ok0 = stage_wait(&bar[0], k.flag, k.wait_ns);
  if (active && ok0) {
    const int sl = row >> 5;
    const int so = __ldg(off + sl);
    const int w = (__ldg(off + sl + 1) - so) >> 5;
    const int loc = so - e0 + (row & 31);
    if (s_col[loc] < 0) active = false;  // long row: fx_long_kernel
    int j = 0;
    for (; active && j + U <= w; j += U) {
      int cj[U];
      uint64_t a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cj[u] = s_col[loc + 32 * (j + u)];
        a[u] = s_val[loc + 32 * (j + u)];
      }
      uint64_t y[U][R];
#pragma unroll
      for (int u = 0; u < U; ++u) load_u64_row<R>(ycur + (size_t)cj[u] * R, y[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        sa += a[u];
#pragma unroll
        for (int c = 0; c < R; ++c) mac(S[c], a[u], y[u][c]);
      }
    }
    for (; active && j < w; ++j) {
      const int cj = s_col[loc + 32 * j];
      const uint64_t a = s_val[loc + 32 * j];
      uint64_t y[R];
      load_u64_row<R>(ycur + (size_t)cj * R, y);
      sa += a;
#pragma unroll
      for (int c = 0; c < R; ++c) mac(S[c], a, y[c]);
    }
  }
  const bool ok1 = vb ? stage_wait(&bar[1], k.flag, k.wait_ns) : true;
  if (active && ok0 && ok1) {
    const size_t idx = (size_t)row * R;
    if (vb) {
      uint64_t own[R], sum[R];
#pragma unroll
      for (int c = 0; c < R; ++c) {
        own[c] = s_own[t * R + c];
        sum[c] = FIRST ? 0ull : s_sum[t * R + c];
      }
      finish_row<R, FIRST, LAST>(idx, S, sa, own, sum, ynext, acc, W, k);
    } else {
      finish_row_global<R, FIRST, LAST>(idx, S, sa, ycur, yprev, ynext, acc, W, k);
    }
  }
  // nothing may still be copying into this CTA's shared memory when it exits
  if (!ok0) tc::mbar_wait_drain(&bar[0], 0);
  if (!ok1) tc::mbar_wait_drain(&bar[1], 0);
}

// CSR rows, one thread per row and all R columns, for rows of at most
// long_row entries (the others are fx_long_kernel's).
template <int R, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads) fx_rows_kernel(int n, int long_row, const int* __restrict__ rowptr,
                                                           const int* __restrict__ col,
                                                           const uint64_t* __restrict__ sval,
                                                           const uint64_t* __restrict__ ycur, const uint64_t* yprev,
                                                           uint64_t* ynext, uint64_t* acc, double* W, FxStep k) {
  allow_dependents();
  const int row = blockIdx.x * kThreads + (int)threadIdx.x;
  if (row >= n) return;
  const int jb = __ldg(rowptr + row), je = __ldg(rowptr + row + 1);
  if (je - jb > long_row) return;
  grid_dependency_wait();
  Acc S[R];
#pragma unroll
  for (int t = 0; t < R; ++t) acc_init(S[t], FIRST ? kValBits + 1 : kValBits);
  uint64_t sa = 0;
  for (int j = jb; j < je; ++j) {
    const int cj = __ldg(col + j);
    const uint64_t a = __ldg(sval + j);
    uint64_t y[R];
    load_u64_row<R>(ycur + (size_t)cj * R, y);
    sa += a;
#pragma unroll
    for (int t = 0; t < R; ++t) mac(S[t], a, y[t]);
  }
  finish_row_global<R, FIRST, LAST>((size_t)row * R, S, sa, ycur, yprev, ynext, acc, W, k);
}

// Rows above long_row entries: one CTA per row, partial sums over strided
// entries combined across the CTA (warp shuffles, then shared memory).
template <int R, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads) fx_long_kernel(const int* __restrict__ long_rows,
                                                           const int* __restrict__ rowptr,
                                                           const int* __restrict__ col,
                                                           const uint64_t* __restrict__ sval,
                                                           const uint64_t* __restrict__ ycur, const uint64_t* yprev,
                                                           uint64_t* ynext, uint64_t* acc, double* W, FxStep k) {
  __shared__ Acc red[kThreads / 32][R];
  __shared__ uint64_t red_sa[kThreads / 32];
  const int row = long_rows[blockIdx.x];
  const int jb = __ldg(rowptr + row), je = __ldg(rowptr + row + 1);
  Acc S[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    S[t].w1 = S[t].w2 = S[t].w3 = 0u;
    S[t].sy = 0ull;
  }
  uint64_t sa = 0;
  for (int j = jb + (int)threadIdx.x; j < je; j += kThreads) {
    const uint64_t a = __ldg(sval + j);
    uint64_t y[R];
    load_u64_row<R>(ycur + (size_t)__ldg(col + j) * R, y);
    sa += a;
#pragma unroll
    for (int t = 0; t < R; ++t) mac(S[t], a, y[t]);
  }
  for (int d = 16; d > 0; d >>= 1) {
    sa += __shfl_down_sync(0xffffffffu, sa, d);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      Acc o;
      o.w1 = __shfl_down_sync(0xffffffffu, S[t].w1, d);
      o.w2 = __shfl_down_sync(0xffffffffu, S[t].w2, d);
      o.w3 = __shfl_down_sync(0xffffffffu, S[t].w3, d);
      o.sy = __shfl_down_sync(0xffffffffu, S[t].sy, d);
      acc_add(S[t], o);
    }
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red_sa[warp] = sa;
#pragma unroll
    for (int t = 0; t < R; ++t) red[warp][t] = S[t];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  Acc T[R];
#pragma unroll
  for (int t = 0; t < R; ++t) acc_init(T[t], FIRST ? kValBits + 1 : kValBits);
  uint64_t ta = 0;
  for (int w = 0; w < kThreads / 32; ++w) {
    ta += red_sa[w];
#pragma unroll
    for (int t = 0; t < R; ++t) acc_add(T[t], red[w][t]);
  }
  finish_row_global<R, FIRST, LAST>((size_t)row * R, T, ta, ycur, yprev, ynext, acc, W, k);
}

// ---- conversions -------------------------------------------------------------
// Per-CTA partial sums of squares of the r columns (fixed order: deterministic).
__global__ void fx_colsq_kernel(const double* __restrict__ V, int64_t n, int r, double* __restrict__ part) {
  __shared__ double red[kThreads / 32][16];
  double s[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) s[t] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
#pragma unroll
    for (int t = 0; t < 16; ++t)
      if (t < r) s[t] = fma(V[i * r + t], V[i * r + t], s[t]);
#pragma unroll
  for (int t = 0; t < 16; ++t)
    for (int d = 16; d > 0; d >>= 1) s[t] += __shfl_down_sync(0xffffffffu, s[t], d);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int t = 0; t < 16; ++t) red[threadIdx.x >> 5][t] = s[t];
  __syncthreads();
  if (threadIdx.x < r) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][threadIdx.x];
    part[(size_t)blockIdx.x * 16 + threadIdx.x] = v;
  }
}

// Column scale exponents: E_t with ||v_t|| <= 2^E_t (1 + 2^-20), least such
// (0 for a zero column).
__global__ void fx_colexp_kernel(const double* __restrict__ part, int parts, int r, int* __restrict__ cexp) {
  const int t = threadIdx.x;
  if (t >= r) return;
  double s = 0.0;
  for (int b = 0; b < parts; ++b) s += part[(size_t)b * 16 + t];
  int e = 0;
  if (s > 0.0) {
    const double nrm = sqrt(s) / (1.0 + 0x1p-20);
    frexp(nrm, &e);  // nrm < 2^e
  }
  cexp[t] = e;
}

// Y = round(V 2^(F - E_t)), offset-binary
__global__ void fx_to_fixed_kernel(const double* __restrict__ V, int64_t count, int r, const int* __restrict__ cexp,
                                   int vec_bits, uint64_t* __restrict__ Y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] = (uint64_t)__double2ll_rn(V[i] * pow2(vec_bits - cexp[i % r])) + kOff;
}

// W = b_0 V for degree 0
__global__ void fx_scale_kernel(const double* __restrict__ V, double* __restrict__ W, double b, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    W[i] = b * V[i];
}

// 2 Ahat = (2/e)(A - cI) in units of 2^-61, offset-binary, for the CSR order
// (sell = false) or the SELL-32 layout; records the largest absolute row sum
// of 2 Ahat (as the bits of a positive FP64, which order like integers).
__global__ void fx_values_kernel(int64_t n, const int* __restrict__ rowptr, const int* __restrict__ diag_pos,
                                 const double* __restrict__ val, int long_row, const int* __restrict__ off, int sell,
                                 double s, double shift, uint64_t* __restrict__ out,
                                 unsigned long long* __restrict__ rowsum_bits) {
  double big = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j0 = rowptr[i], len = rowptr[i + 1] - j0;
    const int d = diag_pos[i];
    double rs = 0.0;
    if (!sell) {
      for (int j = 0; j < len; ++j) {
        const double v = s * (val[j0 + j] - (j0 + j == d ? shift : 0.0));
        rs += fabs(v);
        out[j0 + j] = (uint64_t)__double2ll_rn(v * 0x1p61) + kOff;
      }
    } else {
      const int64_t sl = i >> 5;
      const int base = off[sl] + (int)(i & 31);
      const int w = (off[sl + 1] - off[sl]) >> 5;
      for (int j = 0; j < len; ++j) rs += fabs(s * (val[j0 + j] - (j0 + j == d ? shift : 0.0)));
      for (int j = 0; j < w; ++j) {
        double v = 0.0;
        if (len <= long_row && j < len) v = s * (val[j0 + j] - (j0 + j == d ? shift : 0.0));
        out[base + 32 * j] = (uint64_t)__double2ll_rn(v * 0x1p61) + kOff;
      }
    }
    big = fmax(big, rs);
  }
  for (int d = 16; d > 0; d >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, d));
  if ((threadIdx.x & 31) == 0 && big > 0.0) atomicMax(rowsum_bits, (unsigned long long)__double_as_longlong(big));
}

inline unsigned blocks_for(int64_t count) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 16));
}

// Small device words of the fixed-point path: [8, 16) column exponents, [16]
// the overflow flag, [24] the row-sum maximum; zeroed when first allocated.
void fx_scratch(flz_matrix* A, cudaStream_t st) {
  FxValues& F = A->fx;
  if (F.scratch.p) return;
  F.scratch.reserve(32);
  FLZ_CUDA(cudaMemsetAsync(F.scratch.p, 0, sizeof(uint64_t) * 32, st));
}

// Rows of 2 Ahat may hold absolute sums up to kRowSumLimit (the overflow
// check needs (L + 1) 1.25 < 2^(63-F) = 8 at F = 60; the values need
// |2 Ahat_ij| < 4); up to kRowSumFine the vectors get F = 61 ((L + 1) 1.25 < 4).
constexpr double kRowSumLimit = 3.9;
constexpr double kRowSumFine = 2.1;

// Builds the fixed-point values of 2 Ahat for (c, e) in the layout the
// kernels read (SELL-32, plus CSR order for its long rows; or CSR order), if
// not built yet; false if a row of 2 Ahat has too large an absolute sum for
// the format (the caller then uses FP64 arithmetic).
bool fx_prepare(flz_matrix* A, double c, double e, bool use_sell, cudaStream_t st) {
  FxValues& F = A->fx;
  auto build = [&](int slot) {
    if (F.ok[slot] && F.c[slot] == c && F.e[slot] == e) return;
    DevBuf<uint64_t>& buf = slot ? F.sell : F.csr;
    buf.reserve((size_t)std::max<int64_t>(slot ? A->sell_len : A->nnz, 1));
    unsigned long long* bits_dev = reinterpret_cast<unsigned long long*>(F.scratch.p + 24);
    FLZ_CUDA(cudaMemsetAsync(bits_dev, 0, sizeof(unsigned long long), st));
    fx_values_kernel<<<blocks_for(A->n), 256, 0, st>>>(A->n, A->rowptr.p, A->diag_pos.p, A->val.p, kLongRow,
                                                       A->sell_off.p, slot, 2.0 / e, c, buf.p, bits_dev);
    FLZ_LAUNCH_CHECK();
    unsigned long long bits = 0;
    FLZ_CUDA(cudaMemcpyAsync(&bits, bits_dev, sizeof(bits), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    std::memcpy(&F.rowsum[slot], &bits, sizeof(double));
    F.c[slot] = c;
    F.e[slot] = e;
    F.ok[slot] = true;
  };
  build(use_sell ? 1 : 0);
  if (use_sell && A->n_long > 0) build(0);  // the long rows read the CSR-order values
  return F.rowsum[use_sell ? 1 : 0] <= kRowSumLimit;
}

// Dynamic shared memory of the staged SELL kernel at width R.
size_t sell_stage_bytes(int R, int64_t emax) { return 16 + 2 * (size_t)kThreads * R * 8 + (size_t)emax * 12; }
// Largest stage used; beyond it (SELL slices of very long rows) the CSR row kernel runs instead.
constexpr size_t kMaxStage = 160 * 1024;

template <int R, int U, bool F, bool L>
void set_stage_limit(size_t bytes) {
  static size_t done = 0;
  if (bytes > done) {
    FLZ_CUDA(cudaFuncSetAttribute(fx_sell_kernel<R, U, F, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes));
    done = bytes;
  }
}

template <int R, int U>
void run_fx(const flz_matrix* A, bool sell, const uint64_t* vsell, const uint64_t* vcsr, const uint64_t* b, int m,
            const uint64_t* y0, uint64_t* ya, uint64_t* yb, uint64_t* acc, double* W, const FxStep& base,
            bool vec_bulk, cudaStream_t st) {
  const int n = (int)A->n;
  const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
  const int nsl = (int)((A->n + 31) / 32);
  const int emax = (int)A->sell_cta_entries;
  const size_t smem = sell_stage_bytes(R, emax);
  const int nl = A->n_long;
  const int* lr = A->long_rows.p;
  const int* rp = A->rowptr.p;
  const int* cl = A->col.p;
  const int thr = nl > 0 ? kLongRow : 0x7fffffff;
  const int vb = vec_bulk ? 1 : 0;
  if (sell) {
    set_stage_limit<R, U, true, true>(smem);
    set_stage_limit<R, U, true, false>(smem);
    set_stage_limit<R, U, false, true>(smem);
    set_stage_limit<R, U, false, false>(smem);
  }
  auto step = [&](bool first, bool last, const uint64_t* cur, const uint64_t* prev, uint64_t* next, int k) {
    FxStep s = base;
    s.b_cur = b[0];
    s.b_next = b[k + 1];
#define FX_LAUNCH(F_, L_)                                                                                        \
  do {                                                                                                           \
    if (sell) {                                                                                                  \
      if (F_)                                                                                                    \
        fx_sell_kernel<R, U, F_, L_><<<grid, kThreads, smem, st>>>(n, nsl, emax, vb, A->sell_off.p,              \
                                                                    A->sell_col.p, vsell, cur, prev, next, acc, \
                                                                    W, s);                                       \
      else                                                                                                       \
        launch_dependent(fx_sell_kernel<R, U, F_, L_>, grid, kThreads, smem, st, n, nsl, emax, vb,               \
                         A->sell_off.p, A->sell_col.p, vsell, cur, prev, next, acc, W, s);                       \
    } else {                                                                                                     \
      if (F_)                                                                                                    \
        fx_rows_kernel<R, F_, L_><<<grid, kThreads, 0, st>>>(n, thr, rp, cl, vcsr, cur, prev, next, acc, W, s); \
      else                                                                                                       \
        launch_dependent(fx_rows_kernel<R, F_, L_>, grid, kThreads, 0, st, n, thr, rp, cl, vcsr, cur, prev,      \
                         next, acc, W, s);                                                                       \
    }                                                                                                            \
    FLZ_LAUNCH_CHECK();                                                                                          \
    if (nl) {                                                                                                    \
      fx_long_kernel<R, F_, L_><<<nl, kThreads, 0, st>>>(lr, rp, cl, vcsr, cur, prev, next, acc, W, s);         \
      FLZ_LAUNCH_CHECK();                                                                                        \
    }                                                                                                            \
  } while (0)
    if (first && last) FX_LAUNCH(true, true);
    else if (first) FX_LAUNCH(true, false);
    else if (last) FX_LAUNCH(false, true);
    else FX_LAUNCH(false, false);
#undef FX_LAUNCH
  };
  // step 0 reads Y_0 = V, writes Y_1 to ya; then Y_{k+1} overwrites Y_{k-1}
  step(true, m == 1, y0, nullptr, ya, 0);
  const uint64_t* prev = y0;
  const uint64_t* cur = ya;
  for (int k = 1; k < m; ++k) {
    uint64_t* next = (k == 1) ? yb : const_cast<uint64_t*>(prev);
    step(false, k + 1 == m, cur, prev, next, k);
    prev = cur;
    cur = next;
  }
}

}  // namespace

void fx_fetch_flag(flz_matrix* A, cudaStream_t st);

// Row-per-thread widths of the fixed-point kernels.
bool fx_supported(int r) { return r == 1 || r == 2 || r == 3 || r == 4 || r == 8 || r == 16; }

bool fx_filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int m, int r, const double* V,
                     double* W, cudaStream_t st) {
  const int64_t nr = A->n * (int64_t)r;
  // even widths load and store rows as 16-byte vectors: W (the running sum) must be 16-byte aligned
  if (!fx_supported(r) || (r % 2 == 0 && reinterpret_cast<uintptr_t>(W) % 16 != 0)) return false;
  if (m == 0) {
    fx_scale_kernel<<<blocks_for(nr), 256, 0, st>>>(V, W, coeffs[0], nr);
    FLZ_LAUNCH_CHECK();
    return true;
  }
  fx_scratch(A, st);
  // the staged SELL kernel where its shared-memory stage fits, else CSR rows
  const bool sell = A->sell && sell_stage_bytes(r, A->sell_cta_entries) <= kMaxStage;
  if (!fx_prepare(A, c, e, sell, st)) return false;
  FxValues& F = A->fx;
  const int Fb = F.rowsum[sell ? 1 : 0] <= kRowSumFine ? 61 : 60;
  // coefficients: offset-binary in units of 2^-61, scaled by 2^-s so that the
  // running sum (at most max_k sum_{i<=k} |b_i| times 1.25) stays below
  // 0.9375 2^(63-F), and every |b_i| 2^-s below 3.9 (the units of 2^-61 hold |.| < 4)
  double partial = 0.0, big = 0.0, bmax = 0.0;
  for (int i = 0; i <= m; ++i) {
    partial += std::fabs(coeffs[i]);
    big = std::max(big, partial);
    bmax = std::max(bmax, std::fabs(coeffs[i]));
  }
  int s = 0;
  while (big * 1.25 * std::ldexp(1.0, -s) >= 0.9375 * std::ldexp(1.0, 63 - Fb) || bmax * std::ldexp(1.0, -s) >= 3.9) ++s;
  if (s > 60) return false;
  std::vector<uint64_t> b(m + 1);
  for (int i = 0; i <= m; ++i)
    b[i] = (uint64_t)std::llrint(std::ldexp(coeffs[i], kValBits - s)) + kOff;
  // scratch: Y_0, two recurrence buffers (each 16-byte aligned for the bulk
  // copies); the running sum lives in W
  const int64_t nr2 = (nr + 1) & ~int64_t(1);
  F.ws.reserve(3 * (size_t)nr2);
  uint64_t* y0 = F.ws.p;
  uint64_t* ya = y0 + nr2;
  uint64_t* yb = ya + nr2;
  int* cexp = reinterpret_cast<int*>(F.scratch.p + 8);
  unsigned* flag = reinterpret_cast<unsigned*>(F.scratch.p + 16);
  // the flag reports this application only (an earlier one may have failed
  // without being checked, when another error ended its call first)
  FLZ_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
  const int parts = 152;
  F.part.reserve((size_t)parts * 16);
  fx_colsq_kernel<<<parts, kThreads, 0, st>>>(V, A->n, r, F.part.p);
  FLZ_LAUNCH_CHECK();
  fx_colexp_kernel<<<1, 32, 0, st>>>(F.part.p, parts, r, cexp);
  FLZ_LAUNCH_CHECK();
  fx_to_fixed_kernel<<<blocks_for(nr), 256, 0, st>>>(V, nr, r, cexp, Fb, y0);
  FLZ_LAUNCH_CHECK();
  FxStep base{0, 0, kOff, kOff, 1, cexp, s, Fb, 5ull << (Fb - 2), flag, wait_limit_ns()};
  uint64_t* acc = reinterpret_cast<uint64_t*>(W);
  const uint64_t* vs = F.sell.p;
  const uint64_t* vc = F.csr.p;
  const bool vb = reinterpret_cast<uintptr_t>(W) % 16 == 0;
  switch (r) {
    case 1: run_fx<1, 8>(A, sell, vs, vc, b.data(), m, y0, ya, yb, acc, W, base, vb, st); break;
    case 2: run_fx<2, 8>(A, sell, vs, vc, b.data(), m, y0, ya, yb, acc, W, base, vb, st); break;
    case 3: run_fx<3, 4>(A, sell, vs, vc, b.data(), m, y0, ya, yb, acc, W, base, vb, st); break;
    case 4: run_fx<4, 4>(A, sell, vs, vc, b.data(), m, y0, ya, yb, acc, W, base, vb, st); break;
    case 8: run_fx<8, 2>(A, sell, vs, vc, b.data(), m, y0, ya, yb, acc, W, base, vb, st); break;
    default: run_fx<16, 1>(A, sell, vs, vc, b.data(), m, y0, ya, yb, acc, W, base, vb, st); break;
  }
  fx_fetch_flag(A, st);
  return true;
}

// Copies the overflow flag to pinned host memory the handle owns (valid
// after the next synchronization of st).
void fx_fetch_flag(flz_matrix* A, cudaStream_t st) {
  FxValues& F = A->fx;
  if (!F.scratch.p) return;
  if (!F.flag_host) {
    FLZ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&F.flag_host), sizeof(unsigned)));
    *F.flag_host = 0;
  }
  FLZ_CUDA(cudaMemcpyAsync(F.flag_host, F.scratch.p + 16, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
}

// Raises if a fetched flag was set (and clears it for the next call).
void fx_check_flag(flz_matrix* A) {
  FxValues& F = A->fx;
  if (F.flag_host && *F.flag_host) {
    const unsigned f = *F.flag_host;
    *F.flag_host = 0;
    cudaMemset(F.scratch.p + 16, 0, sizeof(uint64_t));
    if (f & 2u) fail(FLZ_ERR_TIMEOUT, "fixed-point filter: a shared-memory stage wait expired");
    fail(FLZ_ERR_INVALID_ARG,
         "fixed-point filter: a recurrence value left [-1.25, 1.25] of its column scale (the spectrum of "
         "(A - cI)/e is not inside [-1, 1])");
  }
}


// ---- batches ------------------------------------------------------------------
// The same degree step over the block-diagonal concatenation of a batch's
// problems: each row takes its problem's coefficients, sum scaling, degree
// and active flag; a CTA whose rows all belong to finished problems returns
// before staging anything.

namespace {

constexpr int kTileP0 = 128;  // rows per entry of the starting-problem table

struct FxSegArgs {
  int n, nsl, emax, vec_bulk, count;
  const int* off;         // SELL slice offsets of the concatenation
  const int* scol;
  const uint64_t* sval;   // 2 Ahat_i, offset-binary, units 2^-61
  const int* d_off;       // count + 1 problem row offsets
  const int* cta_p0;      // problem of the first row of every kTileP0 rows
  const uint64_t* bfix;   // coefficient table: b_k of problem i at k * count + i
  const int* sexp;        // per-problem sum exponent s_i
  const int* zexp;        // 16 zero column exponents (unit columns)
  const int* mdeg;        // per-problem degree m_i
  const int* active;
  uint64_t* acc;          // running sums (aliases W)
  double* W;
  int vec_bits;
  uint64_t limit;
  unsigned* flag;
  uint64_t wait_ns;
};

__device__ __forceinline__ int seg_problem(const int* __restrict__ d_off, int count, int row) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(d_off + mid) <= row) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ROWS rows (ROWS / 32 SELL slices) per CTA, 128 or 256: a tile shape the
// batch autotuner times.
template <int R, int U, bool FIRST, int ROWS>
__global__ void __launch_bounds__(ROWS, (R <= 4 ? 4 : (R <= 8 ? 2 : 1)) * (256 / ROWS))
    fx_seg_sell_kernel(FxSegArgs a, int k, const uint64_t* __restrict__ ycur, const uint64_t* yprev, uint64_t* ynext) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);         // [0] matrix range, [1] vector rows
  uint64_t* s_own = reinterpret_cast<uint64_t*>(smem + 32);  // V (first step) or Y_{k-1} rows
  uint64_t* s_sum = s_own + ROWS * R;                        // running-sum rows
  uint64_t* s_val = s_sum + ROWS * R;
  int* s_col = reinterpret_cast<int*>(s_val + a.emax);
  const int row0 = blockIdx.x * ROWS, rows = min(ROWS, a.n - row0);
  // the row's problem: forward from the CTA's first row's (rows of a CTA
  // span one or a few problems)
  const int t = threadIdx.x, row = row0 + t;
  int pi = 0, md = 0;
  bool active = row < a.n;
  if (active) {
    pi = __ldg(a.cta_p0 + blockIdx.x * (ROWS / kTileP0));
    while (pi + 1 < a.count && __ldg(a.d_off + pi + 1) <= row) ++pi;
    md = __ldg(a.mdeg + pi);
    active = __ldg(a.active + pi) && k + 1 <= md;
  }
  if (!__syncthreads_or(active)) return;  // reads nothing the previous degree writes
  const int sl0 = blockIdx.x * (ROWS / 32), sl1 = min(a.nsl, sl0 + ROWS / 32);
  const int e0 = __ldg(a.off + sl0), e1 = __ldg(a.off + sl1);
  const bool vb = a.vec_bulk && ((rows * R) % 2 == 0);  // uniform over the CTA
  // the running sums are staged on the regular flush steps; a problem whose
  // last degree falls between them reads its rows' sums directly
  const bool regular = !FIRST && flush_terms(k + 1, false) > 0;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
    tc::mbar_expect_tx(&bar[0], (uint32_t)(e1 - e0) * 12u);
    tc::bulk_g2s(s_val, a.sval + e0, (uint32_t)(e1 - e0) * 8u, &bar[0]);
    tc::bulk_g2s(s_col, a.scol + e0, (uint32_t)(e1 - e0) * 4u, &bar[0]);
  }
  __syncthreads();
  allow_dependents();
  grid_dependency_wait();  // the vectors below are the previous degree's output
  if (threadIdx.x == 0 && vb) {
    const uint32_t bytes = (uint32_t)rows * R * 8u;
    const size_t at = (size_t)row0 * R;
    if (FIRST) {
      tc::mbar_expect_tx(&bar[1], bytes);
      tc::bulk_g2s(s_own, ycur + at, bytes, &bar[1]);
    } else {
      tc::mbar_expect_tx(&bar[1], regular ? 2 * bytes : bytes);
      tc::bulk_g2s(s_own, yprev + at, bytes, &bar[1]);
      if (regular) tc::bulk_g2s(s_sum, a.acc + at, bytes, &bar[1]);
    }
  }
  Acc S[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc_init(S[c], FIRST ? kValBits + 1 : kValBits);
  uint64_t sa = 0;
  const bool ok0 = stage_wait(&bar[0], a.flag, a.wait_ns);
  if (active && ok0) {
    const int sl = row >> 5;
    const int so = __ldg(a.off + sl);
    const int w = (__ldg(a.off + sl + 1) - so) >> 5;
    const int loc = so - e0 + (row & 31);
    int j = 0;
    for (; j + U <= w; j += U) {
      int cj[U];
      uint64_t av[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cj[u] = s_col[loc + 32 * (j + u)];
        av[u] = s_val[loc + 32 * (j + u)];
      }
      uint64_t y[U][R];
#pragma unroll
      for (int u = 0; u < U; ++u) load_u64_row<R>(ycur + (size_t)cj[u] * R, y[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        sa += av[u];
#pragma unroll
        for (int c = 0; c < R; ++c) mac(S[c], av[u], y[u][c]);
      }
    }
    for (; j < w; ++j) {
      const int cj = s_col[loc + 32 * j];
      const uint64_t av = s_val[loc + 32 * j];
      uint64_t y[R];
      load_u64_row<R>(ycur + (size_t)cj * R, y);
      sa += av;
#pragma unroll
      for (int c = 0; c < R; ++c) mac(S[c], av, y[c]);
    }
  }
  const bool ok1 = vb ? stage_wait(&bar[1], a.flag, a.wait_ns) : true;
  if (active && ok0 && ok1) {
    const size_t idx = (size_t)row * R;
    const bool last = k + 1 == md;
    FxStep ks{FIRST ? __ldg(a.bfix + pi) : kOff, __ldg(a.bfix + (size_t)(k + 1) * a.count + pi),
              FIRST ? kOff : __ldg(a.bfix + (size_t)k * a.count + pi),
              k >= 1 ? __ldg(a.bfix + (size_t)(k - 1) * a.count + pi) : kOff, k + 1, a.zexp, __ldg(a.sexp + pi),
              a.vec_bits, a.limit, a.flag, a.wait_ns};
    const bool need_sum = !FIRST && flush_terms(k + 1, last) > 0;
    uint64_t own[R], sum[R];
#pragma unroll
    for (int c = 0; c < R; ++c) sum[c] = 0ull;
    if (vb) {
#pragma unroll
      for (int c = 0; c < R; ++c) own[c] = s_own[t * R + c];
      if (need_sum && regular) {
#pragma unroll
        for (int c = 0; c < R; ++c) sum[c] = s_sum[t * R + c];
      } else if (need_sum) {
        load_u64_row<R>(a.acc + idx, sum);
      }
    } else {
      load_u64_row<R>((FIRST ? ycur : yprev) + idx, own);
      if (need_sum) load_u64_row<R>(a.acc + idx, sum);
    }
    if (last) finish_row_flush3<R, FIRST, true>(idx, S, sa, own, sum, ycur, ynext, a.acc, a.W, ks);
    else finish_row_flush3<R, FIRST, false>(idx, S, sa, own, sum, ycur, ynext, a.acc, a.W, ks);
  }
  // nothing may still be copying into this CTA's shared memory when it exits
  if (!ok0) tc::mbar_wait_drain(&bar[0], 0);
  if (!ok1) tc::mbar_wait_drain(&bar[1], 0);
}

// Y_0 = round(Q_j 2^F), offset-binary (unit columns: column exponent 0)
__global__ void fx_seg_load_kernel(const double* __restrict__ Q, const int* __restrict__ jdev, int64_t nr, int vec_bits,
                                   uint64_t* __restrict__ y0) {
  const double* src = Q + (size_t)(*jdev) * nr;
  const double sc = pow2(vec_bits);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x)
    y0[i] = (uint64_t)__double2ll_rn(src[i] * sc) + kOff;
}

// 2 Ahat_i in the SELL-32 layout of the concatenation, each row in its
// problem's map; records the largest absolute row sum.
__global__ void fx_seg_values_kernel(int64_t n, const int* __restrict__ rowptr, const int* __restrict__ diag_pos,
                                     const double* __restrict__ val, const int* __restrict__ off,
                                     const int* __restrict__ d_off, int count, const double* __restrict__ cc,
                                     const double* __restrict__ ee, uint64_t* __restrict__ out,
                                     unsigned long long* __restrict__ rowsum_bits) {
  double big = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int pi = seg_problem(d_off, count, (int)i);
    const double s = 2.0 / ee[pi], shift = cc[pi];
    const int j0 = rowptr[i], len = rowptr[i + 1] - j0, d = diag_pos[i];
    const int64_t sl = i >> 5;
    const int base = off[sl] + (int)(i & 31);
    const int w = (off[sl + 1] - off[sl]) >> 5;
    double rs = 0.0;
    for (int j = 0; j < w; ++j) {
      double v = 0.0;
      if (j < len) v = s * (val[j0 + j] - (j0 + j == d ? shift : 0.0));
      rs += fabs(v);
      out[base + 32 * j] = (uint64_t)__double2ll_rn(v * 0x1p61) + kOff;
    }
    big = fmax(big, rs);
  }
  for (int d = 16; d > 0; d >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, d));
  if ((threadIdx.x & 31) == 0 && big > 0.0) atomicMax(rowsum_bits, (unsigned long long)__double_as_longlong(big));
}

// ---- the persistent variant: every degree in one cooperative launch ----
// The grid (all CTAs resident: a cooperative launch) walks the 256-row tiles
// of the concatenation for degree 0, meets at a grid barrier, walks them for
// degree 1, and so on. No shared-memory staging: the vectors another CTA
// wrote in the previous degree are read through L2 (__ldcg), the constant
// matrix through the read-only path. The barrier is bounded: a CTA that waits
// longer than wait_ns sets bit 2 of the flag (a timeout) and leaves, and the
// others then time out at their next barrier; nothing spins without limit.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, uint64_t wait_ns,
                                             unsigned* flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = *reinterpret_cast<volatile unsigned*>(gen);
    __threadfence();  // this CTA's writes of the degree before its arrival
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *reinterpret_cast<volatile unsigned*>(count) = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const uint64_t t0 = tc::globaltimer();
      while (*reinterpret_cast<volatile unsigned*>(gen) == g) {
        if (wait_ns == 0 || tc::globaltimer() - t0 > wait_ns) {
          atomicOr(flag, 2u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int R, int U>
__device__ __forceinline__ void seg_tile_plain(const FxSegArgs& a, int k, int tile, const uint64_t* ycur,
                                               const uint64_t* yprev, uint64_t* ynext) {
  const bool first = k == 0;
  const int row = tile * kThreads + (int)threadIdx.x;
  if (row >= a.n) return;
  int pi = __ldg(a.cta_p0 + tile * (kThreads / kTileP0));
  while (pi + 1 < a.count && __ldg(a.d_off + pi + 1) <= row) ++pi;
  const int md = __ldg(a.mdeg + pi);
  if (!__ldg(a.active + pi) || k + 1 > md) return;
  const int sl = row >> 5;
  const int so = __ldg(a.off + sl);
  const int w = (__ldg(a.off + sl + 1) - so) >> 5;
  const int base = so + (row & 31);
  Acc S[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc_init(S[c], first ? kValBits + 1 : kValBits);
  uint64_t sa = 0;
  int j = 0;
  for (; j + U <= w; j += U) {
    int cj[U];
    uint64_t av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cj[u] = __ldg(a.scol + base + 32 * (j + u));
      av[u] = __ldg(a.sval + base + 32 * (j + u));
    }
    uint64_t y[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) load_u64_row_cg<R>(ycur + (size_t)cj[u] * R, y[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      sa += av[u];
#pragma unroll
      for (int c = 0; c < R; ++c) mac(S[c], av[u], y[u][c]);
    }
  }
  for (; j < w; ++j) {
    const int cj = __ldg(a.scol + base + 32 * j);
    const uint64_t av = __ldg(a.sval + base + 32 * j);
    uint64_t y[R];
    load_u64_row_cg<R>(ycur + (size_t)cj * R, y);
    sa += av;
#pragma unroll
    for (int c = 0; c < R; ++c) mac(S[c], av, y[c]);
  }
  const size_t idx = (size_t)row * R;
  const bool last = k + 1 == md;
  FxStep ks{first ? __ldg(a.bfix + pi) : kOff, __ldg(a.bfix + (size_t)(k + 1) * a.count + pi),
            first ? kOff : __ldg(a.bfix + (size_t)k * a.count + pi),
            k >= 1 ? __ldg(a.bfix + (size_t)(k - 1) * a.count + pi) : kOff, k + 1, a.zexp, __ldg(a.sexp + pi),
            a.vec_bits, a.limit, a.flag, a.wait_ns};
  uint64_t own[R], sum[R];
#pragma unroll
  for (int c = 0; c < R; ++c) sum[c] = 0ull;
  load_u64_row_cg<R>((first ? ycur : yprev) + idx, own);
  if (!first && flush_terms(k + 1, last) > 0) load_u64_row_cg<R>(a.acc + idx, sum);
  if (first) {
    if (last) finish_row_flush3<R, true, true, true>(idx, S, sa, own, sum, ycur, ynext, a.acc, a.W, ks);
    else finish_row_flush3<R, true, false, true>(idx, S, sa, own, sum, ycur, ynext, a.acc, a.W, ks);
  } else {
    if (last) finish_row_flush3<R, false, true, true>(idx, S, sa, own, sum, ycur, ynext, a.acc, a.W, ks);
    else finish_row_flush3<R, false, false, true>(idx, S, sa, own, sum, ycur, ynext, a.acc, a.W, ks);
  }
}

template <int R, int U>
__global__ void __launch_bounds__(kThreads, R <= 4 ? 4 : (R <= 8 ? 2 : 1))
    fx_seg_persistent_kernel(FxSegArgs a, int mmax, const uint64_t* y0, uint64_t* ya, uint64_t* yb, unsigned* gbar) {
  const int ntiles = (a.n + kThreads - 1) / kThreads;
  const uint64_t* prev = nullptr;
  const uint64_t* cur = y0;
  uint64_t* next = ya;
  for (int k = 0; k < mmax; ++k) {
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) seg_tile_plain<R, U>(a, k, tile, cur, prev, next);
    if (k + 1 < mmax && !grid_barrier(gbar, gbar + 1, gridDim.x, a.wait_ns, a.flag)) return;
    uint64_t* nn = (k == 0) ? yb : const_cast<uint64_t*>(prev);
    prev = cur;
    cur = next;
    next = nn;
  }
}

template <int R, int U>
void run_fx_seg_persistent(FxBatch& F, const FxSegArgs& a, cudaStream_t st) {
  static int per_sm = -1;
  if (per_sm < 0) {
    FLZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fx_seg_persistent_kernel<R, U>, kThreads, 0));
    if (per_sm < 1) fail(FLZ_ERR_CUDA, "persistent batch kernel: no resident CTA");
  }
  int dev = 0, sms = 0;
  FLZ_CUDA(cudaGetDevice(&dev));
  FLZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int ntiles = (int)((F.n + kThreads - 1) / kThreads);
  const int grid = std::max(1, std::min(ntiles, per_sm * sms));
  FxSegArgs args = a;
  int mmax = F.mmax;
  const uint64_t* y0 = F.y0.p;
  uint64_t* ya = F.ya.p;
  uint64_t* yb = F.yb.p;
  unsigned* gbar = F.gbar.p;
  void* params[] = {&args, &mmax, &y0, &ya, &yb, &gbar};
  // a barrier an earlier launch left early (a timeout) must not count its arrivals here
  FLZ_CUDA(cudaMemsetAsync(gbar, 0, sizeof(unsigned), st));
  FLZ_CUDA(cudaLaunchCooperativeKernel((const void*)fx_seg_persistent_kernel<R, U>, dim3(grid), dim3(kThreads),
                                       params, 0, st));
  FLZ_LAUNCH_CHECK();
}

// emax: the most entries of any 8 consecutive slices (256 rows), which bounds
// those of 4 slices too
size_t seg_stage_bytes(int R, int64_t emax, int rows = 256) { return 32 + 2 * (size_t)rows * R * 8 + (size_t)emax * 12; }

template <int R, int U, bool FIRST, int ROWS>
void seg_stage_limit(size_t bytes) {
  static size_t done = 0;
  if (bytes > done) {
    FLZ_CUDA(cudaFuncSetAttribute(fx_seg_sell_kernel<R, U, FIRST, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes));
    done = bytes;
  }
}

template <int R, int U, int ROWS>
void run_fx_seg_rows(FxBatch& F, const FxSegArgs& a, bool pdl, cudaStream_t st) {
  const unsigned grid = (unsigned)((F.n + ROWS - 1) / ROWS);
  const size_t smem = seg_stage_bytes(R, F.emax, ROWS);
  seg_stage_limit<R, U, true, ROWS>(smem);
  seg_stage_limit<R, U, false, ROWS>(smem);
  fx_seg_sell_kernel<R, U, true, ROWS><<<grid, ROWS, smem, st>>>(a, 0, F.y0.p, nullptr, F.ya.p);
  FLZ_LAUNCH_CHECK();
  const uint64_t* prev = F.y0.p;
  const uint64_t* cur = F.ya.p;
  for (int k = 1; k < F.mmax; ++k) {
    uint64_t* next = (k == 1) ? F.yb.p : const_cast<uint64_t*>(prev);
    if (pdl)
      launch_dependent(fx_seg_sell_kernel<R, U, false, ROWS>, grid, ROWS, smem, st, a, k, cur, prev, next);
    else
      fx_seg_sell_kernel<R, U, false, ROWS><<<grid, ROWS, smem, st>>>(a, k, cur, prev, next);
    FLZ_LAUNCH_CHECK();
    prev = cur;
    cur = next;
  }
}

template <int R, int U>
void run_fx_seg(FxBatch& F, const FxSegArgs& a, bool pdl, cudaStream_t st) {
  if (F.rows == 128) run_fx_seg_rows<R, U, 128>(F, a, pdl, st);
  else run_fx_seg_rows<R, U, 256>(F, a, pdl, st);
}

}  // namespace

bool fx_batch_prepare(FxBatch& F, int64_t N, int64_t nnz, const int* rowptr, const int* col, const double* val,
                      const int* diag_pos, int32_t max_row_nnz, const int* d_off, const std::vector<int>& off_host,
                      int count, const double* cc, const double* ee, int r, cudaStream_t st) {
  if (!fx_supported(r) || max_row_nnz > kLongRow) return false;
  if (!F.layout_built) {
    // the problem of every CTA's first row
    const int64_t ctas = (N + kTileP0 - 1) / kTileP0;
    std::vector<int> p0(ctas);
    int p = 0;
    for (int64_t b = 0; b < ctas; ++b) {
      while (p + 1 < count && (int64_t)off_host[p + 1] <= b * kTileP0) ++p;
      p0[b] = p;
    }
    F.cta_p0.reserve((size_t)ctas);
    FLZ_CUDA(cudaMemcpy(F.cta_p0.p, p0.data(), sizeof(int) * ctas, cudaMemcpyHostToDevice));
    F.layout_built = true;
    F.layout_ok = false;
    flz_matrix tmp;  // borrows the concatenation's structure to build its SELL-32 layout
    tmp.n = N;
    tmp.nnz = nnz;
    tmp.rowptr.p = const_cast<int*>(rowptr);
    tmp.col.p = const_cast<int*>(col);
    build_sell(&tmp);
    tmp.rowptr.p = nullptr;
    tmp.col.p = nullptr;
    if (tmp.sell) {
      std::swap(F.sell_off.p, tmp.sell_off.p);
      std::swap(F.sell_off.count, tmp.sell_off.count);
      std::swap(F.sell_col.p, tmp.sell_col.p);
      std::swap(F.sell_col.count, tmp.sell_col.count);
      F.n = N;
      F.nsl = (N + 31) / 32;
      F.emax = tmp.sell_cta_entries;
      F.sval.reserve((size_t)std::max<int64_t>(tmp.sell_len, 1));
      F.zexp.reserve(16);
      FLZ_CUDA(cudaMemset(F.zexp.p, 0, sizeof(int) * 16));
      F.flag.reserve(2);
      FLZ_CUDA(cudaMemset(F.flag.p, 0, sizeof(unsigned) * 2));
      F.gbar.reserve(2);  // grid-barrier arrival count and generation
      FLZ_CUDA(cudaMemset(F.gbar.p, 0, sizeof(unsigned) * 2));
      FLZ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&F.flag_host), sizeof(unsigned)));
      *F.flag_host = 0;
      F.layout_ok = true;
    }
  }
  if (!F.layout_ok || seg_stage_bytes(r, F.emax) > kMaxStage) return false;
  F.count = count;
  unsigned long long* bits_dev = reinterpret_cast<unsigned long long*>(F.flag.p);  // the flag words, reused
  FLZ_CUDA(cudaMemsetAsync(bits_dev, 0, sizeof(unsigned long long), st));
  fx_seg_values_kernel<<<blocks_for(N), 256, 0, st>>>(N, rowptr, diag_pos, val, F.sell_off.p, d_off, count, cc, ee,
                                                      F.sval.p, bits_dev);
  FLZ_LAUNCH_CHECK();
  unsigned long long bits = 0;
  FLZ_CUDA(cudaMemcpyAsync(&bits, bits_dev, sizeof(bits), cudaMemcpyDeviceToHost, st));
  FLZ_CUDA(cudaStreamSynchronize(st));
  FLZ_CUDA(cudaMemsetAsync(bits_dev, 0, sizeof(unsigned long long), st));
  std::memcpy(&F.rowsum, &bits, sizeof(double));
  if (!(F.rowsum <= kRowSumLimit)) return false;
  F.vec_bits = F.rowsum <= kRowSumFine ? 61 : 60;
  const size_t nr2 = ((size_t)N * r + 1) & ~size_t(1);
  F.y0.reserve(nr2);
  F.ya.reserve(nr2);
  F.yb.reserve(nr2);
  return true;
}

bool fx_batch_coefficients(FxBatch& F, const std::vector<std::vector<double>>& coeffs, cudaStream_t st) {
  const int count = (int)coeffs.size();
  int mmax = 0;
  for (const auto& v : coeffs) {
    if (v.size() < 2) return false;  // degree 0: no recurrence step
    mmax = std::max(mmax, (int)v.size() - 1);
  }
  std::vector<uint64_t> table((size_t)(mmax + 1) * count, kOff);
  std::vector<int> sexp(count);
  for (int i = 0; i < count; ++i) {
    // the same scaling as a single application: the running sum below
    // 0.9375 2^(63-F) and every scaled |b_k| below 3.9
    double partial = 0.0, big = 0.0, bmax = 0.0;
    for (double b : coeffs[i]) {
      partial += std::fabs(b);
      big = std::max(big, partial);
      bmax = std::max(bmax, std::fabs(b));
    }
    int sc = 0;
    while (big * 1.25 * std::ldexp(1.0, -sc) >= 0.9375 * std::ldexp(1.0, 63 - F.vec_bits) ||
           bmax * std::ldexp(1.0, -sc) >= 3.9)
      ++sc;
    if (sc > 60) return false;
    sexp[i] = sc;
    for (size_t q = 0; q < coeffs[i].size(); ++q)
      table[q * count + i] = (uint64_t)std::llrint(std::ldexp(coeffs[i][q], kValBits - sc)) + kOff;
  }
  F.mmax = mmax;
  F.bfix.reserve(table.size());
  F.sexp.reserve(count);
  FLZ_CUDA(cudaMemcpyAsync(F.bfix.p, table.data(), sizeof(uint64_t) * table.size(), cudaMemcpyHostToDevice, st));
  FLZ_CUDA(cudaMemcpyAsync(F.sexp.p, sexp.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  FLZ_CUDA(cudaStreamSynchronize(st));  // the host tables go out of scope
  return true;
}

void fx_batch_filter(FxBatch& F, int r, const double* Q, const int* jdev, const int* d_off, const int* mdeg,
                     const int* active, double* W, bool pdl, bool persistent, cudaStream_t st) {
  const int64_t nr = F.n * (int64_t)r;
  fx_seg_load_kernel<<<blocks_for(nr), 256, 0, st>>>(Q, jdev, nr, F.vec_bits, F.y0.p);
  FLZ_LAUNCH_CHECK();
  FxSegArgs a{(int)F.n, (int)F.nsl, (int)F.emax, reinterpret_cast<uintptr_t>(W) % 16 == 0 ? 1 : 0, F.count,
              F.sell_off.p, F.sell_col.p, F.sval.p, d_off, F.cta_p0.p, F.bfix.p, F.sexp.p, F.zexp.p, mdeg, active,
              reinterpret_cast<uint64_t*>(W), W, F.vec_bits, 5ull << (F.vec_bits - 2), F.flag.p, wait_limit_ns()};
  if (persistent) {
    switch (r) {
      case 1: run_fx_seg_persistent<1, 8>(F, a, st); break;
      case 2: run_fx_seg_persistent<2, 8>(F, a, st); break;
      case 4: run_fx_seg_persistent<4, 4>(F, a, st); break;
      case 8: run_fx_seg_persistent<8, 2>(F, a, st); break;
      case 16: run_fx_seg_persistent<16, 1>(F, a, st); break;
      default: fail(FLZ_ERR_INVALID_ARG, "batch block width %d", r);
    }
    return;
  }
  switch (r) {
    case 1: run_fx_seg<1, 8>(F, a, pdl, st); break;
    case 2: run_fx_seg<2, 8>(F, a, pdl, st); break;
    case 4: run_fx_seg<4, 4>(F, a, pdl, st); break;
    case 8: run_fx_seg<8, 2>(F, a, pdl, st); break;
    case 16: run_fx_seg<16, 1>(F, a, pdl, st); break;
    default: fail(FLZ_ERR_INVALID_ARG, "batch block width %d", r);
  }
}

void fx_batch_check_flag(FxBatch& F, cudaStream_t st) {
  if (!F.flag_host) return;
  FLZ_CUDA(cudaMemcpyAsync(F.flag_host, F.flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FLZ_CUDA(cudaStreamSynchronize(st));
  const unsigned f = *F.flag_host;
  if (!f) return;
  *F.flag_host = 0;
  FLZ_CUDA(cudaMemsetAsync(F.flag.p, 0, sizeof(unsigned), st));
  if (f & 2u) fail(FLZ_ERR_TIMEOUT, "batch fixed-point filter: a shared-memory stage wait expired");
  fail(FLZ_ERR_INVALID_ARG, "batch fixed-point filter: a recurrence value left [-1.25, 1.25] (a spectrum of some "
                            "(A_i - c_i I)/e_i is not inside [-1, 1])");
}

}  // namespace flz
