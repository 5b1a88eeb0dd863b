// W = p_m(Ahat) V by the vectorized Clenshaw recurrence of Section 2.2:
//   B_{m+1} = B_{m+2} = 0,
//   B_k = b_k V + 2 Ahat B_{k+1} - B_{k+2}     (k = m, ..., 1),
//   W   = b_0 V + Ahat B_1 - B_2.
// One launch per degree makes one pass over the CSR matrix and four vector
// streams (V, the gathered B_{k+1}, B_{k+2}, and B_k written over B_{k+2}),
// one fewer than the forward recurrence with its running sum, and in the
// BF16 path no FP32 sum stream at all.
//
// With 2 Ahat stored (shift and 2/e folded into the values) every launch has
// the form
//   out = alpha V + g (2 Ahat) X - Z
// where B_m = b_m V is never stored:
//   k = m-1:  X = V,       g = b_m, alpha = b_{m-1},          no Z
//   k = m-2:  X = B_{m-1}, g = 1,   alpha = b_{m-2} - b_m,    no Z
//   k < m-2:  X = B_{k+1}, g = 1,   alpha = b_k,              Z = B_{k+2}
//   final:    X = B_1,     g = 1/2, alpha = b_0 (- b_2 if m = 2), Z = B_2 (m >= 3)
// and m = 1 is the single launch W = b_0 V + (b_1/2)(2 Ahat) V.
// For g = 1 the row sum is seeded with alpha V - Z, so a degree costs the
// same multiply-adds as the forward recurrence.
#include <type_traits>

#include "device_common.cuh"
#include "flz_internal.h"

namespace flz {

using namespace dev;

namespace {

constexpr int kRows = 256;  // rows (threads) per CTA in the row kernel
constexpr int kLanes = 256;

// One Clenshaw launch with one thread per row (all R columns). The CTA's CSR
// range is staged in shared memory when it fits `cap` entries, as in the
// forward kernel. UNIT: g == 1 (seeded row sum). Z may be null (uniform).
// out may alias z (same element, same thread); x never aliases out.
template <int R, class MS, class VS, class OutS, bool UNIT>
__global__ void __launch_bounds__(kRows) clen_rows_kernel(
    int n, int cap, int long_row, const int* __restrict__ rowptr, const int* __restrict__ col,
    const MS* __restrict__ sval, const VS* __restrict__ x, const VS* __restrict__ v, const VS* z, OutS* out,
    typename Arith<VS>::type alpha, typename Arith<VS>::type g) {
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
  if (je - jb > long_row) return;  // rows longer than long_row belong to clen_long_kernel
  grid_dependency_wait();  // B_{k+1}, B_{k+2} are earlier launches' output
  A base[R];
  load_row<VS, R>(v + (size_t)row * R, base);
#pragma unroll
  for (int t = 0; t < R; ++t) base[t] = alpha * base[t];
  if (z) {
    A zz[R];
    load_row<VS, R>(z + (size_t)row * R, zz);
#pragma unroll
    for (int t = 0; t < R; ++t) base[t] = base[t] - zz[t];
  }
  A s[R];
#pragma unroll
  for (int t = 0; t < R; ++t) s[t] = UNIT ? base[t] : A(0);
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
    for (int u = 0; u < U; ++u) load_row<VS, R>(x + (size_t)cj[u] * R, y[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < R; ++t) s[t] = fma(a[u], y[u][t], s[t]);
  }
  for (; j < je; ++j) {
    const int cj = staged ? s_col[j - j0] : __ldg(col + j);
    const A a = staged ? to_arith(s_val[j - j0]) : to_arith(sval[j]);
    A y[R];
    load_row<VS, R>(x + (size_t)cj * R, y);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = fma(a, y[t], s[t]);
  }
  if (!UNIT) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = fma(g, s[t], base[t]);
  }
  if constexpr (std::is_same<OutS, VS>::value) {
    store_row_rounded<VS, R>(out + (size_t)row * R, s);
  } else {
    store_acc<R>(out + (size_t)row * R, s);
  }
}

// The same launch on the SELL-32 layout (see cheb_sell_kernel): coalesced,
// independent loads of a row's indices and values, no staging.
template <int R, class MS, class VS, class OutS, bool UNIT>
__global__ void __launch_bounds__(kRows) clen_sell_kernel(
    int n, const int* __restrict__ off, const int* __restrict__ scol, const MS* __restrict__ sval,
    const VS* __restrict__ x, const VS* __restrict__ v, const VS* z, OutS* out, typename Arith<VS>::type alpha,
    typename Arith<VS>::type g) {
  using A = typename Arith<VS>::type;
  allow_dependents();
  const int row = blockIdx.x * kRows + (int)threadIdx.x;
  if (row >= n) return;
  const int sl = row >> 5;
  const int o = __ldg(off + sl);
  const int w = (__ldg(off + sl + 1) - o) >> 5;
  const int base = o + (row & 31);
  if (__ldg(scol + base) < 0) return;  // long row: clen_long_kernel
  grid_dependency_wait();  // B_{k+1}, B_{k+2} are earlier launches' output
  A base_v[R];
  load_row<VS, R>(v + (size_t)row * R, base_v);
#pragma unroll
  for (int t = 0; t < R; ++t) base_v[t] = alpha * base_v[t];
  if (z) {
    A zz[R];
    load_row<VS, R>(z + (size_t)row * R, zz);
#pragma unroll
    for (int t = 0; t < R; ++t) base_v[t] = base_v[t] - zz[t];
  }
  A s[R];
#pragma unroll
  for (int t = 0; t < R; ++t) s[t] = UNIT ? base_v[t] : A(0);
  sell_row_sum<R, MS, VS, A>(scol, sval, base, w, x, s);
  if (!UNIT) {
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = fma(g, s[t], base_v[t]);
  }
  if constexpr (std::is_same<OutS, VS>::value) {
    store_row_rounded<VS, R>(out + (size_t)row * R, s);
  } else {
    store_acc<R>(out + (size_t)row * R, s);
  }
}

// The same launch for rows with more than `long_row` entries: one CTA per
// row, strided entries, tree reduction in shared memory.
template <int R, class MS, class VS, class OutS>
__global__ void __launch_bounds__(kRows) clen_long_kernel(
    const int* __restrict__ long_rows, const int* __restrict__ rowptr, const int* __restrict__ col,
    const MS* __restrict__ sval, const VS* __restrict__ x, const VS* __restrict__ v, const VS* z, OutS* out,
    typename Arith<VS>::type alpha, typename Arith<VS>::type g) {
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
    load_row<VS, R>(x + (size_t)__ldg(col + j) * R, y);
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
  A res[R], vv[R];
  load_row<VS, R>(v + (size_t)row * R, vv);
#pragma unroll
  for (int t = 0; t < R; ++t) res[t] = fma(g, red[t * kRows], alpha * vv[t]);
  if (z) {
    A zz[R];
    load_row<VS, R>(z + (size_t)row * R, zz);
#pragma unroll
    for (int t = 0; t < R; ++t) res[t] = res[t] - zz[t];
  }
  if constexpr (std::is_same<OutS, VS>::value) {
    store_row_rounded<VS, R>(out + (size_t)row * R, res);
  } else {
    store_acc<R>(out + (size_t)row * R, res);
  }
}

// Lane-per-column form for block widths without an aligned R-wide path
// (r = 3, 5, ...): r consecutive lanes own one row.
template <class MS, class VS, class OutS>
__global__ void __launch_bounds__(kLanes) clen_lanes_kernel(
    int n, int r, int rows_per_warp, const int* __restrict__ rowptr, const int* __restrict__ col,
    const MS* __restrict__ sval, const VS* __restrict__ x, const VS* __restrict__ v, const VS* z, OutS* out,
    typename Arith<VS>::type alpha, typename Arith<VS>::type g) {
  using A = typename Arith<VS>::type;
  const int lane = threadIdx.x & 31;
  const int sub = lane / r;
  const int c = lane - sub * r;
  const long long warp = ((long long)blockIdx.x * kLanes + threadIdx.x) >> 5;
  const long long row = warp * rows_per_warp + sub;
  if (sub >= rows_per_warp || row >= n) return;
  const size_t idx = (size_t)row * r + c;
  A s = A(0);
  int j = __ldg(rowptr + row);
  const int jend = __ldg(rowptr + row + 1);
  for (; j + 4 <= jend; j += 4) {
    const int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2), c3 = __ldg(col + j + 3);
    const A a0 = to_arith(sval[j]), a1 = to_arith(sval[j + 1]), a2 = to_arith(sval[j + 2]), a3 = to_arith(sval[j + 3]);
    const A y0 = to_arith(x[(size_t)c0 * r + c]);
    const A y1 = to_arith(x[(size_t)c1 * r + c]);
    const A y2 = to_arith(x[(size_t)c2 * r + c]);
    const A y3 = to_arith(x[(size_t)c3 * r + c]);
    s = fma(a0, y0, s);
    s = fma(a1, y1, s);
    s = fma(a2, y2, s);
    s = fma(a3, y3, s);
  }
  for (; j < jend; ++j) s = fma(to_arith(sval[j]), to_arith(x[(size_t)__ldg(col + j) * r + c]), s);
  A res = fma(g, s, alpha * to_arith(v[idx]));
  if (z) res = res - to_arith(z[idx]);
  if constexpr (std::is_same<OutS, VS>::value) {
    out[idx] = from_arith<VS>(res);
  } else {
    out[idx] = store_as<OutS>(res);
  }
}

// One Clenshaw launch: out = alpha V + g (2 Ahat) X - Z, over all rows.
struct Launch {
  const void* x;
  const void* z;
  void* out;
  double alpha, g;
  bool unit, to_w;
  bool dependent;  // follows another launch of this recurrence on the stream
};

template <int R, class MS, class VS, class WT>
void launch_rows(const flz_matrix* A, const MS* vsell, const MS* val, const VS* v, const Launch& L, cudaStream_t st) {
  using Ar = typename Arith<VS>::type;
  const int n = (int)A->n;
  const int cap = std::min<int>(A->max_cta_nnz, 4096);
  const size_t smem = vsell ? 0 : (size_t)cap * (sizeof(MS) + sizeof(int));
  const unsigned grid = (unsigned)((n + kRows - 1) / kRows);
  const int nl = A->n_long;
  const int thr = nl > 0 ? kLongRow : 0x7fffffff;
  const VS* x = static_cast<const VS*>(L.x);
  const VS* z = static_cast<const VS*>(L.z);
  const Ar al = Ar(L.alpha), g = Ar(L.g);
  const int* rp = A->rowptr.p;
  const int* cl = A->col.p;
  const int* of = A->sell_off.p;
  const int* sc = A->sell_col.p;
  // one launch of the row kernel (SELL-32 or staged CSR), as a programmatic
  // dependent launch when it follows another launch of this recurrence
  auto go = [&](auto out, auto unit_tag) {
    using O = std::remove_pointer_t<decltype(out)>;
    constexpr bool U = decltype(unit_tag)::value;
    if (vsell) {
      if (L.dependent)
        launch_dependent(clen_sell_kernel<R, MS, VS, O, U>, grid, kRows, 0, st, n, of, sc, vsell, x, v, z, out, al, g);
      else
        clen_sell_kernel<R, MS, VS, O, U><<<grid, kRows, 0, st>>>(n, of, sc, vsell, x, v, z, out, al, g);
    } else {
      if (L.dependent)
        launch_dependent(clen_rows_kernel<R, MS, VS, O, U>, grid, kRows, smem, st, n, cap, thr, rp, cl, val, x, v, z,
                         out, al, g);
      else
        clen_rows_kernel<R, MS, VS, O, U><<<grid, kRows, smem, st>>>(n, cap, thr, rp, cl, val, x, v, z, out, al, g);
    }
    FLZ_LAUNCH_CHECK();
    if (nl) {
      clen_long_kernel<R, MS, VS, O><<<nl, kRows, 0, st>>>(A->long_rows.p, rp, cl, val, x, v, z, out, al, g);
      FLZ_LAUNCH_CHECK();
    }
  };
  if (L.to_w)
    go(static_cast<WT*>(L.out), std::false_type{});
  else if (L.unit)
    go(static_cast<VS*>(L.out), std::true_type{});
  else
    go(static_cast<VS*>(L.out), std::false_type{});
}

template <class MS, class VS, class WT>
void launch_lanes(const flz_matrix* A, const MS* val, int r, const VS* v, const Launch& L, cudaStream_t st) {
  using Ar = typename Arith<VS>::type;
  const int n = (int)A->n;
  const int rpw = 32 / r;
  const int64_t warps = (n + rpw - 1) / rpw;
  const unsigned grid = (unsigned)((warps * 32 + kLanes - 1) / kLanes);
  const VS* x = static_cast<const VS*>(L.x);
  const VS* z = static_cast<const VS*>(L.z);
  const Ar al = Ar(L.alpha), g = Ar(L.g);
  if (L.to_w) {
    clen_lanes_kernel<MS, VS, WT><<<grid, kLanes, 0, st>>>(n, r, rpw, A->rowptr.p, A->col.p, val, x, v, z,
                                                           static_cast<WT*>(L.out), al, g);
  } else {
    clen_lanes_kernel<MS, VS, VS><<<grid, kLanes, 0, st>>>(n, r, rpw, A->rowptr.p, A->col.p, val, x, v, z,
                                                           static_cast<VS*>(L.out), al, g);
  }
  FLZ_LAUNCH_CHECK();
}

inline bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

template <class MS, class VS, class WT>
void run_clenshaw(const flz_matrix* A, const MS* vsell, const MS* val, const double* b, int m, int r, const VS* v,
                  VS* ba, VS* bb, WT* W, cudaStream_t st) {
  const bool pow2 = row_kernel_width(r) && r != 3;  // r = 3: SELL-32 or the lane kernel
  const size_t av = row_alignment(r, sizeof(VS));
  const size_t aw = row_alignment(r, sizeof(WT));
  const bool rows = vsell || (pow2 && A->max_cta_nnz > 0 && aligned_to(v, av) && aligned_to(ba, av) &&
                              aligned_to(bb, av) && aligned_to(W, aw));
  auto go = [&](const Launch& L) {
    if (!rows) {
      launch_lanes<MS, VS, WT>(A, val, r, v, L, st);
      return;
    }
    switch (r) {
      case 1: launch_rows<1, MS, VS, WT>(A, vsell, val, v, L, st); break;
      case 2: launch_rows<2, MS, VS, WT>(A, vsell, val, v, L, st); break;
      case 3: launch_rows<3, MS, VS, WT>(A, vsell, val, v, L, st); break;
      case 4: launch_rows<4, MS, VS, WT>(A, vsell, val, v, L, st); break;
      case 8: launch_rows<8, MS, VS, WT>(A, vsell, val, v, L, st); break;
      default: launch_rows<16, MS, VS, WT>(A, vsell, val, v, L, st); break;
    }
  };
  if (m == 1) {
    go({v, nullptr, W, b[0], 0.5 * b[1], false, true, false});
    return;
  }
  // B_{m-1} = b_{m-1} V + b_m (2 Ahat) V
  go({v, nullptr, ba, b[m - 1], b[m], false, false, false});
  const VS* cur = ba;   // B_{k+1}
  VS* prev = nullptr;   // B_{k+2} (B_m = b_m V is implicit)
  for (int k = m - 2; k >= 1; --k) {
    VS* out;
    if (k == m - 2) {
      out = bb;
      go({cur, nullptr, out, b[k] - b[m], 1.0, true, false, true});
    } else {
      out = prev;  // B_k overwrites B_{k+2}
      go({cur, prev, out, b[k], 1.0, true, false, true});
    }
    prev = const_cast<VS*>(cur);
    cur = out;
  }
  if (m == 2) {
    go({cur, nullptr, W, b[0] - b[2], 0.5, false, true, true});
  } else {
    go({cur, prev, W, b[0], 0.5, false, true, true});
  }
}

#define FLZ_CLENSHAW_INST(MS, VS, WT)                                                                         \
  template void run_clenshaw<MS, VS, WT>(const flz_matrix*, const MS*, const MS*, const double*, int, int, const VS*, \
                                         VS*, VS*, WT*, cudaStream_t);
FLZ_CLENSHAW_INST(double, double, double)
FLZ_CLENSHAW_INST(float, float, double)
FLZ_CLENSHAW_INST(__nv_bfloat16, __nv_bfloat16, double)
FLZ_CLENSHAW_INST(dfloat, dfloat, double)
FLZ_CLENSHAW_INST(dfloat, dfloat, dfloat)

}  // namespace flz
