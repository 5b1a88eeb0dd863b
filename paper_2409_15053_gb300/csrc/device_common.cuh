// Device helpers shared by the filter kernels: the arithmetic type of each
// storage type, conversions, and R-wide row loads/stores (one thread owns a
// whole row of an n x R row-major block).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

namespace flz {
namespace dev {

using ::fma;  // the dfloat overload below joins the built-in ones, it must not hide them

// Double-FP32 number hi + lo (|lo| <= ulp(hi)/2): about 48 significant bits
// carried in two FP32 words and combined on the FP32 pipes with error-free
// transformations (TwoSum, Knuth; TwoProduct via FMA, Ogita-Rump-Oishi).
struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

#if defined(__CUDACC__)

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfloat(s, e);
}
__device__ __forceinline__ dfloat quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// a * b + c
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const dfloat s = two_sum(p, c.hi);
  const float lo = __fadd_rn(__fadd_rn(s.lo, e), c.lo);
  return quick_two_sum(s.hi, lo);
}
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return fma(a, b, dfloat(0.f, 0.f)); }
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const dfloat s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + dfloat(-b.hi, -b.lo); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }
__device__ __forceinline__ double to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic
// stream serialization may start while its predecessor drains. It must not
// read anything the predecessor writes before grid_dependency_wait(), which
// returns once the predecessor has completed and its writes are visible (a
// no-op for a normal launch). allow_dependents() lets the next kernel be
// scheduled once every CTA of this grid has started.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <class S>
struct Arith {
  using type = float;
};
template <>
struct Arith<double> {
  using type = double;
};
template <>
struct Arith<dfloat> {
  using type = dfloat;
};

__device__ __forceinline__ double to_arith(double x) { return x; }
__device__ __forceinline__ float to_arith(float x) { return x; }
__device__ __forceinline__ float to_arith(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ dfloat to_arith(dfloat x) { return x; }

template <class S>
__device__ __forceinline__ S from_arith(typename Arith<S>::type x);
template <>
__device__ __forceinline__ double from_arith<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_arith<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_arith<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ dfloat from_arith<dfloat>(dfloat x) { return x; }

template <class O, class A>
__device__ __forceinline__ O store_as(A x) { return static_cast<O>(x); }

// ---- R-wide row I/O: one thread owns a whole row of an n x R block ----------
template <class S, int R>
struct RowIO;

template <int R>
struct RowIO<double, R> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {  // one element at a time (odd widths: no aligned vectors)
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = p[i];
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 2) {
        const double2 t = *reinterpret_cast<const double2*>(p + i);
        v[i] = t.x;
        v[i + 1] = t.y;
      }
    }
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) p[i] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 2) *reinterpret_cast<double2*>(p + i) = make_double2(v[i], v[i + 1]);
    }
  }
};

template <int R>
struct RowIO<float, R> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = p[i];
    } else if constexpr (R == 2) {
      const float2 t = *reinterpret_cast<const float2*>(p);
      v[0] = t.x;
      v[1] = t.y;
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 4) {
        const float4 t = *reinterpret_cast<const float4*>(p + i);
        v[i] = t.x;
        v[i + 1] = t.y;
        v[i + 2] = t.z;
        v[i + 3] = t.w;
      }
    }
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) p[i] = v[i];
    } else if constexpr (R == 2) {
      *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 4) *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
  }
};

template <int R>
struct RowIO<dfloat, R> {
  static __device__ __forceinline__ void load(const dfloat* p, dfloat (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const float2 t = *reinterpret_cast<const float2*>(p + i);
        v[i] = dfloat(t.x, t.y);
      }
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 2) {
        const float4 t = *reinterpret_cast<const float4*>(p + i);
        v[i] = dfloat(t.x, t.y);
        v[i + 1] = dfloat(t.z, t.w);
      }
    }
  }
  static __device__ __forceinline__ void store(dfloat* p, const dfloat (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) *reinterpret_cast<float2*>(p + i) = make_float2(v[i].hi, v[i].lo);
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 2)
        *reinterpret_cast<float4*>(p + i) = make_float4(v[i].hi, v[i].lo, v[i + 1].hi, v[i + 1].lo);
    }
  }
};

template <int R>
struct RowIO<__nv_bfloat16, R> {
  // loads/stores R bf16 values widened to / narrowed from float
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, float (&v)[R]) {
    if constexpr (R == 1 || (R & (R - 1)) != 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = __bfloat162float(p[i]);
    } else if constexpr (R == 2) {
      const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
      v[0] = t.x;
      v[1] = t.y;
    } else if constexpr (R == 4) {
      const uint2 u = *reinterpret_cast<const uint2*>(p);
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
      const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 8) {
        const uint4 u = *reinterpret_cast<const uint4*>(p + i);
        const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[q]));
          v[i + 2 * q] = f.x;
          v[i + 2 * q + 1] = f.y;
        }
      }
    }
  }
  // rounds to bf16, stores, and returns the rounded values in v
  static __device__ __forceinline__ void store(__nv_bfloat16* p, float (&v)[R]) {
    if constexpr (R != 1 && (R & (R - 1)) != 0) {  // odd widths: element by element, rounded values back in v
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v[i]);
        p[i] = h;
        v[i] = __bfloat162float(h);
      }
    } else {
      store_pow2(p, v);
    }
  }
  // rounds to bf16, stores, and returns the rounded values in v (R a power of two)
  static __device__ __forceinline__ void store_pow2(__nv_bfloat16* p, float (&v)[R]) {
    __nv_bfloat162 h[(R + 1) / 2];
#pragma unroll
    for (int i = 0; i < R; i += 2) {
      h[i / 2] = __floats2bfloat162_rn(v[i], i + 1 < R ? v[i + 1] : 0.f);
      const float2 f = __bfloat1622float2(h[i / 2]);
      v[i] = f.x;
      if (i + 1 < R) v[i + 1] = f.y;
    }
    if constexpr (R == 1) {
      p[0] = h[0].x;
    } else if constexpr (R == 2) {
      *reinterpret_cast<__nv_bfloat162*>(p) = h[0];
    } else if constexpr (R == 4) {
      uint2 u;
      u.x = *reinterpret_cast<unsigned*>(&h[0]);
      u.y = *reinterpret_cast<unsigned*>(&h[1]);
      *reinterpret_cast<uint2*>(p) = u;
    } else {
#pragma unroll
      for (int i = 0; i < R; i += 8) {
        uint4 u;
        u.x = *reinterpret_cast<unsigned*>(&h[i / 2]);
        u.y = *reinterpret_cast<unsigned*>(&h[i / 2 + 1]);
        u.z = *reinterpret_cast<unsigned*>(&h[i / 2 + 2]);
        u.w = *reinterpret_cast<unsigned*>(&h[i / 2 + 3]);
        *reinterpret_cast<uint4*>(p + i) = u;
      }
    }
  }
};

template <class S, int R>
__device__ __forceinline__ void store_row_rounded(S* p, typename Arith<S>::type (&v)[R]) {
  if constexpr (std::is_same<S, __nv_bfloat16>::value) {
    RowIO<S, R>::store(p, v);
  } else {
    RowIO<S, R>::store(p, v);  // FP64 / FP32 storage is the arithmetic type: no rounding
  }
}

template <class S, int R>
__device__ __forceinline__ void load_row(const S* p, typename Arith<S>::type (&v)[R]) {
  RowIO<S, R>::load(p, v);
}

// Running-sum output row: FP64 W (the last launch) or the working sum type.
template <int R, class A>
__device__ __forceinline__ void store_acc(double* p, const A (&v)[R]) {
  double d[R];
#pragma unroll
  for (int t = 0; t < R; ++t) d[t] = (double)v[t];
  RowIO<double, R>::store(p, d);
}
template <int R>
__device__ __forceinline__ void store_acc(float* p, const float (&v)[R]) {
  float f[R];
#pragma unroll
  for (int t = 0; t < R; ++t) f[t] = v[t];
  RowIO<float, R>::store(p, f);
}
template <int R, class A>
__device__ __forceinline__ void load_acc(const double* p, A (&v)[R]) {
  double d[R];
  RowIO<double, R>::load(p, d);
#pragma unroll
  for (int t = 0; t < R; ++t) v[t] = (A)d[t];
}
template <int R>
__device__ __forceinline__ void load_acc(const float* p, float (&v)[R]) {
  RowIO<float, R>::load(p, v);
}
template <int R>
__device__ __forceinline__ void store_acc(double* p, const dfloat (&v)[R]) {
  double d[R];
#pragma unroll
  for (int t = 0; t < R; ++t) d[t] = to_double(v[t]);
  RowIO<double, R>::store(p, d);
}
template <int R>
__device__ __forceinline__ void store_acc(dfloat* p, const dfloat (&v)[R]) {
  RowIO<dfloat, R>::store(p, v);
}
template <int R>
__device__ __forceinline__ void load_acc(const dfloat* p, dfloat (&v)[R]) {
  RowIO<dfloat, R>::load(p, v);
}

// Row sum s[t] += sum_j (2 Ahat)_{row, j} X[j, t] over one row of the SELL-32
// layout: entry j of the row sits at base + 32 j (base = slice offset + lane),
// so a warp's loads of column indices and values are coalesced and
// independent of each other; U entries are in flight per thread.
template <int R, class MS, class VS, class A>
__device__ __forceinline__ void sell_row_sum(const int* __restrict__ scol, const MS* __restrict__ sval, int base,
                                             int w, const VS* __restrict__ x, A (&s)[R]) {
  // entries in flight per thread: 8 for rows up to 16 bytes and for FP64 rows
  // up to 32 bytes, 4 for double-FP32 32-byte rows (measured: 8 was 9 %
  // slower there, 1.5 % faster for FP64), 2 beyond
  constexpr int kRowBytes = R * (int)sizeof(A);
  constexpr int U = kRowBytes <= 16 ? 8 : (kRowBytes <= 32 ? (std::is_same<A, double>::value ? 8 : 4) : 2);
  int j = 0;
  for (; j + U <= w; j += U) {
    int cj[U];
    A a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cj[u] = __ldg(scol + base + 32 * (j + u));
      a[u] = to_arith(sval[base + 32 * (j + u)]);
    }
    A y[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) load_row<VS, R>(x + (size_t)cj[u] * R, y[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < R; ++t) s[t] = fma(a[u], y[u][t], s[t]);
  }
  for (; j < w; ++j) {
    const int cj = __ldg(scol + base + 32 * j);
    const A a = to_arith(sval[base + 32 * j]);
    A y[R];
    load_row<VS, R>(x + (size_t)cj * R, y);
#pragma unroll
    for (int t = 0; t < R; ++t) s[t] = fma(a, y[t], s[t]);
  }
}

#endif  // __CUDACC__

}  // namespace dev
}  // namespace flz
