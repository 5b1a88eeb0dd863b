// Full reorthogonalization (classical Gram-Schmidt twice, Section 3.2.2) on
// the tensor cores, with results at least as accurate as FP64 arithmetic.
//
// Number format. Every basis value x (|x| <= 1 in an orthonormal basis) is
// rounded to the 64-bit fixed-point integer v = round(x 2^62) and split into
// eight balanced base-256 digits, v = sum_s d_s 256^(7-s), d_1..d_7 in
// [-128, 127] and |d_0| <= 66 (<= 123 for any |x| < 1.9). Each digit is an
// integer that BF16 holds exactly. The FP64 basis itself is replaced by
// v 2^-62 (exact in FP64), so the two copies are the same numbers. A block W
// (or a coefficient matrix H) is split the same way after scaling each column
// by 2^(62-E), 2^E the smallest power of two above the column's largest
// magnitude; W's digits are built once per projection by a pre-pass.
//
// Exact products. The product of two digits is at most 2^14 in magnitude, so
// a BF16 x BF16 tensor-core accumulation over at most 256 terms stays below
// 2^22 and is an exact integer in the FP32 accumulator. Both kernels drain
// the tensor-memory accumulators after at most 256 terms into integer
// registers and recombine the 64 digit pairs d_s e_t 256^(14-s-t) in integer
// and FP64 arithmetic. The inner products are therefore exact up to the final
// rounding and the rounding of W to 62 fractional bits of its scale.
//
// Layout of the digit copy (`q`): groups of 16 basis columns; in a group, 16
// strips mg = 2 s + c/8 (s the digit, c the column in the group), each strip
// the whole row range as 8-row x 8-column core matrices of 128 bytes:
//   byte ((G 16 + mg) n_oct + i/8) 128 + (c % 8) 16 + (i % 8) 2.
// A 128-row chunk of one group is 16 strips of 2 KB, each contiguous, moved
// by the bulk-copy (TMA) engine into shared memory where it is both the
// K-major A operand of the projection (M = digit x column, K = rows) and the
// MN-major A operand of the update (M = rows, K = columns).
#include <cstring>

#include "flz_internal.h"
#include "tcgen05.cuh"

namespace flz {

namespace {

constexpr int kDig = 8;              // digits per value
constexpr int kRange = 256;          // rows per exact projection range
constexpr int kChunk = 128;          // rows per staged chunk
constexpr int kWindowGroups = 16;    // groups (256 columns) per exact update window
constexpr int kStrip = kChunk / 8 * 128;  // 2048 bytes: one strip of a chunk
constexpr int kAStage = 16 * kStrip;      // 32 KB: all strips of a group's chunk
constexpr int kUpdStages = 4;
// Shared memory the update kernel reserves past its last stage: its A
// descriptors reach at most 32 KB past a stage under either reading of the
// leading/strided byte-offset fields, so every operand fetch stays inside the
// CTA's allocation whatever the hardware's convention.
constexpr int kUpdPad = 32 * 1024;

// status codes written by the kernels (first failure wins)
constexpr int kErrWaitProducer = 1, kErrWaitMma = 2, kErrWaitEpilogue = 4;

__device__ __forceinline__ double pow2i(int e) {  // 2^e, -1022 <= e <= 1023
  return __longlong_as_double((long long)(e + 1023) << 52);
}
// upper word of |x| (monotone in |x|), the per-column maximum is kept as this
__device__ __forceinline__ uint32_t abs_hiword(double x) {
  return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
}
// E with |x| < 2^E for every x whose upper word is at most hi
__device__ __forceinline__ int scale_exponent(uint32_t hi) {
  if (hi == 0) return 0;
  const int E = (int)((hi >> 20) & 0x7FF) - 1022;
  return min(max(E, -960), 1000);
}
// The balanced base-256 digits of v (most significant first, d_1..d_7 in
// [-128, 127]) as BF16 bit patterns, on full-rate integer and FP32 pipes:
// adding 128 to every base-256 position turns the balanced digits into the
// bytes of one 64-bit sum (no carries: each d_s + 128 is in [0, 255] for
// |v| < 1.9 2^62); d = byte - 128 becomes an exact FP32 through the
// 1.5 * 2^23 offset, whose upper 16 bits are its BF16 (d has at most 8
// significant bits).
__device__ __forceinline__ void digit_bits(long long v, uint32_t (&b)[kDig]) {
  const unsigned long long u = (unsigned long long)v + 0x8080808080808080ull;
#pragma unroll
  for (int s = 0; s < kDig; ++s) {
    const int d = (int)((u >> (8 * (kDig - 1 - s))) & 0xFFu) - 128;
    b[s] = __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
  }
}
// an FP32 accumulator value that is an integer of magnitude <= 2^22, as int
__device__ __forceinline__ int exact_int(uint32_t bits) {
  return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}
// |p| < 2^51 to FP64, exactly, on the integer and FP64 add pipes
__device__ __forceinline__ double small_ll_to_double(long long p) {
  return __longlong_as_double(0x4338000000000000LL + p) - 6755399441055744.0;
}

// ---------------------------------------------------------------------------
// Per-column maxima of an n x r block (as upper words); out pre-zeroed.
__global__ void colmax_kernel(const double* __restrict__ X, int64_t n, int r, int ld, uint32_t* out) {
  uint32_t m[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) m[j] = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < r) m[j] = max(m[j], abs_hiword(X[i * ld + j]));
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t w = __reduce_max_sync(0xffffffffu, m[j]);
    if ((threadIdx.x & 31) == 0 && j < r && w) atomicMax(out + j, w);
  }
}

// Rounds block X (n x r, row stride r) to 62 fractional bits in place and
// writes its digits as basis columns col0 .. col0 + r - 1. One thread per
// (8-row octet, column).
__global__ void basis_digits_kernel(double* __restrict__ X, int64_t n, int r, int col0, uint8_t* __restrict__ q,
                                    int64_t n_oct) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_oct * r) return;
  const int j = (int)(t % r);
  const int64_t o = t / r;
  const int col = col0 + j, G = col >> 4, c = col & 15;
  uint32_t pack[kDig][4];
#pragma unroll
  for (int s = 0; s < kDig; ++s) pack[s][0] = pack[s][1] = pack[s][2] = pack[s][3] = 0u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t i = o * 8 + k;
    long long v = 0;
    if (i < n) {
      const double x = X[i * r + j];
      v = __double2ll_rn(x * 4611686018427387904.0);  // 2^62
      X[i * r + j] = __ll2double_rn(v) * 2.168404344971009e-19;  // 2^-62, exact
    }
    uint32_t bits[kDig];
    digit_bits(v, bits);
#pragma unroll
    for (int s = 0; s < kDig; ++s) pack[s][k >> 1] |= bits[s] << (16 * (k & 1));
  }
#pragma unroll
  for (int s = 0; s < kDig; ++s) {
    uint8_t* dst = q + ((size_t)(G * 16 + 2 * s + (c >> 3)) * n_oct + o) * 128 + (c & 7) * 16;
    *reinterpret_cast<uint4*>(dst) = make_uint4(pack[s][0], pack[s][1], pack[s][2], pack[s][3]);
  }
}

// ---------------------------------------------------------------------------
// Digits of W for the projection, one image per 256-row range exactly as the
// projection stages it in shared memory: the K-major B operand N = NP (column
// j of W, digit t) x K = 256 rows as core matrices (j, row octet o) of 8
// digits x 8 rows: byte rr WSLOT + ((j 32 + o) 8 + t) 16 + (i % 8) 2, WSLOT =
// NP 512. Columns j >= r are zero. One thread per (row octet, column block).
__global__ void w_digits_kernel(const double* __restrict__ W, int64_t n, int r, int ldw, const uint32_t* wmax,
                                int np, int64_t n_oct, uint8_t* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nj = np / 8;
  if (t >= n_oct * nj) return;
  const int j = (int)(t % nj);
  const int64_t og = t / nj, rr = og / (kRange / 8);
  const int o = (int)(og % (kRange / 8));
  uint32_t pack[kDig][4];
#pragma unroll
  for (int s = 0; s < kDig; ++s) pack[s][0] = pack[s][1] = pack[s][2] = pack[s][3] = 0u;
  if (j < r) {
    const double sc = pow2i(62 - scale_exponent(wmax[j]));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t i = og * 8 + k;
      const long long v = i < n ? __double2ll_rn(W[i * ldw + j] * sc) : 0;
      uint32_t b[kDig];
      digit_bits(v, b);
#pragma unroll
      for (int s = 0; s < kDig; ++s) pack[s][k >> 1] |= b[s] << (16 * (k & 1));
    }
  }
  uint8_t* dst = out + (size_t)rr * np * kRange * 2 + (size_t)((j * (kRange / 8) + o) * 8) * 16;
#pragma unroll
  for (int s = 0; s < kDig; ++s)
    *reinterpret_cast<uint4*>(dst + s * 16) = make_uint4(pack[s][0], pack[s][1], pack[s][2], pack[s][3]);
}

// Projection C = Q^T W on the tensor cores.
//
// CTA (x, y): group set x (GPC groups of 16 columns), row ranges y, y + RS,
// ... of 256 rows; the group sets of one range split run side by side, so
// the W digits of a range come from HBM once and from L2 for the others. Per
// range, one bulk copy of its W digits (NP x 256); per 128-row chunk and
// group, one stage of 32 KB (the group's 16 strips). MMA: M = 128 (digit s,
// column c), N = NP (column j of W, digit t), K = 16 rows, 16 instructions
// per range and group into a double-buffered tensor-memory accumulator. The
// epilogue warps add each drained range (exact integers <= 2^22) into int32
// registers (<= 256 ranges per CTA, so <= 2^30) and add those once per CTA
// into 64-bit integer accumulators in global memory (reductions without a
// return value).
struct DotArgs {
  const uint8_t* q;
  const uint8_t* wd;  // W digits, one NP x 256 image per range
  int64_t n_oct;
  int Gtot, nR, RS;
  unsigned long long* acc;  // Gtot x 128 x NP integer sums, zero on entry
  int* status;
  uint64_t wait_ns;         // limit of each barrier wait
};

// stages of the projection's ring: three when the W digits of N = 128 take 128 KB
__host__ __device__ constexpr int dot_stages(int np) { return np == 128 ? 3 : 4; }

template <int NP>
__global__ void __launch_bounds__(192, 1) tc_dot_kernel(DotArgs a) {
  constexpr int GPC = 128 / NP;
  constexpr int kDotStages = dot_stages(NP);
  constexpr int WSLOT = NP * kRange * 2;  // bytes of one range's W digits
  constexpr uint32_t IDESC = tc::idesc_bf16(128, NP, 0, 0);
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sW = smem + kDotStages * kAStage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sW + 2 * WSLOT);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + kDotStages;
  uint64_t* w_full = bars + 2 * kDotStages;
  uint64_t* w_empty = w_full + 2;
  uint64_t* acc_full = w_empty + 2;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(fin + 1);
  int* s_abort = reinterpret_cast<int*>(s_tmem + 1);
  int* s_issued = s_abort + 1;
  int* s_consumed = s_abort + 2;
  int* s_wissued = s_abort + 3;
  int* s_wconsumed = s_abort + 4;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gs = blockIdx.x, split = blockIdx.y;
  const int gcount = min(GPC, a.Gtot - gs * GPC);
  const int nloc = split < a.nR ? (a.nR - 1 - split) / a.RS + 1 : 0;
  const tc::Guard guard{s_abort, a.status, a.wait_ns};

  if (tid == 0) {
    for (int i = 0; i < kDotStages; ++i) {
      tc::mbar_init(a_full + i, 1);
      tc::mbar_init(a_empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(w_full + i, 1);
      tc::mbar_init(w_empty + i, 1);
      tc::mbar_init(acc_full + i, 1);
      tc::mbar_init(acc_empty + i, 128);
    }
    tc::mbar_init(fin, 1);
    *s_abort = 0;
    *s_issued = *s_consumed = *s_wissued = *s_wconsumed = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, 2 * GPC * NP);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;

  if (warp == 0 && lane == 0) {
    // ---- producer: bulk copies of the W digits and the basis digit strips ----
    int k = 0, li = 0;
    for (; li < nloc && !*s_abort; ++li) {
      const int64_t rr = split + (int64_t)li * a.RS;
      const int wslot = li & 1;
      if (li >= 2 && !tc::mbar_wait(w_empty + wslot, ((li >> 1) - 1) & 1, guard, kErrWaitProducer)) break;
      tc::mbar_expect_tx(w_full + wslot, WSLOT);
      tc::bulk_g2s(sW + wslot * WSLOT, a.wd + (size_t)rr * WSLOT, WSLOT, w_full + wslot);
      *s_wissued = li + 1;
      for (int h = 0; h < 2; ++h)
        for (int g = 0; g < gcount; ++g, ++k) {
          const int stage = k % kDotStages, u = k / kDotStages;
          if (u >= 1 && !tc::mbar_wait(a_empty + stage, (u - 1) & 1, guard, kErrWaitProducer)) goto produced;
          tc::mbar_expect_tx(a_full + stage, kAStage);
          const int G = gs * GPC + g;
          const int64_t o0 = rr * (kRange / 8) + h * (kChunk / 8);
          for (int mg = 0; mg < 16; ++mg)
            tc::bulk_g2s(sA + stage * kAStage + mg * kStrip, a.q + ((size_t)(G * 16 + mg) * a.n_oct + o0) * 128,
                         kStrip, a_full + stage);
          *s_issued = k + 1;
        }
    }
  produced:;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int k = 0;
    for (int li = 0; li < nloc; ++li) {
      const int buf = li & 1;
      if (li >= 2 && !tc::mbar_wait(acc_empty + buf, ((li >> 1) - 1) & 1, guard, kErrWaitMma)) break;
      if (!tc::mbar_wait(w_full + buf, (li >> 1) & 1, guard, kErrWaitMma)) break;
      *s_wconsumed = li + 1;
      tc::fence_after_sync();
      const uint32_t wbase = tc::smem_u32(sW + buf * WSLOT);
      bool ok = true;
      for (int h = 0; h < 2 && ok; ++h)
        for (int g = 0; g < gcount; ++g, ++k) {
          const int stage = k % kDotStages, u = k / kDotStages;
          if (!tc::mbar_wait(a_full + stage, u & 1, guard, kErrWaitMma)) {
            ok = false;
            break;
          }
          *s_consumed = k + 1;
          tc::fence_after_sync();
          const uint32_t abase = tc::smem_u32(sA + stage * kAStage);
          const uint32_t d = tmem + (uint32_t)(buf * GPC * NP + g * NP);
#pragma unroll
          for (int ks = 0; ks < kChunk / 16; ++ks) {
            // A: K-major, core matrices 128 B apart along K (rows), strips along M
            const uint64_t ad = tc::smem_desc(abase + ks * 256, 128, kStrip);
            // B: K-major, octets 128 B apart along K, column blocks (8 digits) along N
            const uint64_t bd = tc::smem_desc(wbase + (h * 16 + ks * 2) * 128, 128, (kRange / 8) * 128);
            tc::mma_bf16(d, ad, bd, IDESC, (h | ks) != 0);
          }
          tc::mma_commit(a_empty + stage);
        }
      if (!ok) break;
      tc::mma_commit(w_empty + buf);
      tc::mma_commit(acc_full + buf);
    }
    tc::mma_commit(fin);
  } else if (warp >= 2) {
    // ---- epilogue: drain each range into int32 sums ----
    const int q4 = warp & 3;
    int acc[GPC][NP];
#pragma unroll
    for (int g = 0; g < GPC; ++g)
#pragma unroll
      for (int x = 0; x < NP; ++x) acc[g][x] = 0;
    for (int li = 0; li < nloc; ++li) {
      const int buf = li & 1;
      // warp-uniform outcome: the tensor-memory loads below are .sync.aligned
      if (!__all_sync(0xffffffffu, tc::mbar_wait(acc_full + buf, (li >> 1) & 1, guard, kErrWaitEpilogue))) break;
      tc::fence_after_sync();
#pragma unroll
      for (int g = 0; g < GPC; ++g) {
        if (g < gcount) {
          const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * GPC * NP + g * NP);
          if constexpr (NP == 16) {
            uint32_t v[16];
            tc::tmem_ld16(taddr, v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int x = 0; x < 16; ++x) acc[g][x] += exact_int(v[x]);
          } else {
#pragma unroll
            for (int c = 0; c < NP / 32; ++c) {
              uint32_t v[32];
              tc::tmem_ld32(taddr + 32 * c, v);
              tc::tmem_ld_wait();
#pragma unroll
              for (int x = 0; x < 32; ++x) acc[g][32 * c + x] += exact_int(v[x]);
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(acc_empty + buf);
    }
    const int m = q4 * 32 + lane;
    if (nloc > 0) {
#pragma unroll
      for (int g = 0; g < GPC; ++g) {
        if (g < gcount) {
          const int G = gs * GPC + g;
          unsigned long long* dst = a.acc + ((size_t)G * 128 + m) * NP;
#pragma unroll
          for (int x = 0; x < NP; ++x)  // two's-complement sums: exact for |total| < 2^63
            if (acc[g][x]) atomicAdd(dst + x, (unsigned long long)(long long)acc[g][x]);
        }
      }
    }
  }

  // ---- teardown: nothing in flight may outlive the CTA's shared or tensor memory ----
  __syncthreads();
  if (tid == 0) {
    tc::mbar_wait_drain(fin, 0);  // every MMA this CTA issued has completed
    for (int k = *s_consumed; k < *s_issued; ++k)  // copies issued but never consumed (abort only)
      tc::mbar_wait_drain(a_full + (k % kDotStages), (k / kDotStages) & 1);
    for (int li = *s_wconsumed; li < *s_wissued; ++li)
      tc::mbar_wait_drain(w_full + (li & 1), (li >> 1) & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * GPC * NP);
  }
}

// Reads group G's integer sums (and clears them for the next projection),
// recombines the 64 digit pairs (diagonal by diagonal, exact until the last
// few FP64 additions) and writes C[kb, j] for the group's columns kb < K.
// One thread per (column c of the group, column j of W): 16 r threads.
template <int NP>
__global__ void tc_dot_reduce_kernel(unsigned long long* __restrict__ acc, int K, int r, const uint32_t* wmax,
                                     double* C, int ldc) {
  const int G = blockIdx.x, t = threadIdx.x;
  if (t >= 16 * r) return;
  const int c = t / r, j = t - c * r, kb = G * 16 + c;
  unsigned long long* src = acc + (size_t)G * 128 * NP;
  double S[2 * kDig - 1];
#pragma unroll
  for (int d = 0; d < 2 * kDig - 1; ++d) S[d] = 0.0;
#pragma unroll
  for (int s = 0; s < kDig; ++s)
#pragma unroll
    for (int u = 0; u < kDig; ++u) {
      unsigned long long* e = src + (16 * s + c) * NP + j * 8 + u;
      S[s + u] += (double)(long long)*e;  // |sum| <= (CTAs) 2^30: exact, and so are the diagonal sums
      *e = 0ull;
    }
  if (kb >= K) return;
  double v = S[2 * kDig - 2];
#pragma unroll
  for (int d = 2 * kDig - 3; d >= 0; --d) v = v * 0.00390625 + S[d];
  C[(size_t)kb * ldc + j] = v * pow2i(scale_exponent(wmax[j]) - 12);
}

// Digits of the coefficient matrix H (K x r, row stride ldc) for the update:
// per group G, the K-major B operand N = NP (column j, digit t) x K = 16
// (column c of the group) as core matrices (j, c/8) of 8 digits x 8 columns:
//   halfword G NP 16 + ((j 2 + c/8) 8 + t) 8 + c % 8.
// Also writes the column scale exponents. sign = -1 stores the digits of -H.
__global__ void tc_hdigits_kernel(const double* __restrict__ C, int ldc, int K, int r, int Gtot, int NP,
                                  uint16_t* __restrict__ hs, int* hexp, int sign) {
  __shared__ uint32_t mx[16];
  if (threadIdx.x < 16) mx[threadIdx.x] = 0u;
  __syncthreads();
  for (int e = threadIdx.x; e < K * r; e += blockDim.x) {
    const int kb = e / r, j = e - kb * r;
    atomicMax(&mx[j], abs_hiword(C[(size_t)kb * ldc + j]));
  }
  __syncthreads();
  const int ng = NP / 8;
  for (int e = threadIdx.x; e < Gtot * 16 * ng; e += blockDim.x) {
    const int G = e / (16 * ng), rem = e - G * 16 * ng;
    const int j = rem / 16, c = rem - j * 16, kb = G * 16 + c;
    long long v = 0;
    if (j < r && kb < K) v = sign * __double2ll_rn(C[(size_t)kb * ldc + j] * pow2i(62 - scale_exponent(mx[j])));
    uint32_t bits[kDig];
    digit_bits(v, bits);
#pragma unroll
    for (int t = 0; t < kDig; ++t)
      hs[(size_t)G * NP * 16 + ((j * 2 + (c >> 3)) * 8 + t) * 8 + (c & 7)] = (uint16_t)bits[t];
  }
  if (threadIdx.x < r) hexp[threadIdx.x] = scale_exponent(mx[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Update W -= Q H on the tensor cores, for the columns of groups G0 .. G1-1
// (at most 16 groups: <= 256 terms per exact accumulation).
//
// Persistent CTAs over 128-row tiles. Per tile and group one stage (the 16
// strips, 32 KB, plus the group's H digits, NP x 16); per stage 8 MMAs, one
// per basis digit s: M = 128 rows (A MN-major: strip pair 2s, 2s+1), N = NP
// (column j, digit t), K = 16 columns, into accumulator s of a set of 8
// (two sets, double-buffered, when 16 NP <= 512 tensor-memory columns, i.e.
// up to 4 columns of W; one set for 5..8). The epilogue warps (one row per
// thread) sum the digit pairs by diagonal s + t <= 8 in int32, combine the
// diagonals exactly into three integers below 2^43 and subtract the FP64
// result from W, or (keep = 0) store its negative.
struct UpdArgs {
  const uint8_t* q;
  int64_t n_oct, n;
  int ntiles, G0, G1;
  const uint16_t* hs;
  const int* hexp;
  double* W;
  int r, ldw;
  int keep;            // 1: W -= Q H; 0: W = -Q H (H the digits' value)
  uint32_t* wmax_out;  // per-column maxima of the updated W, or null
  int* status;
  uint64_t wait_ns;    // limit of each barrier wait
};

template <int NP>
__global__ void __launch_bounds__(192, 1) tc_update_kernel(UpdArgs a) {
  constexpr int HB = NP * 32;  // bytes of a group's H digits
  constexpr int STAGE = kAStage + HB;
  constexpr uint32_t IDESC = tc::idesc_bf16(128, NP, 1, 0);
  // two accumulator sets when they fit the 512 tensor-memory columns, else one
  constexpr int NBUF = 2 * kDig * NP <= 512 ? 2 : 1;
  constexpr int NCOL = NBUF * kDig * NP;
  constexpr int NJ = NP / 8;  // columns of W per launch
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kUpdStages * STAGE + kUpdPad);
  uint64_t* full = bars;
  uint64_t* empty = bars + kUpdStages;
  uint64_t* acc_full = bars + 2 * kUpdStages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(fin + 1);
  int* s_abort = reinterpret_cast<int*>(s_tmem + 1);
  int* s_issued = s_abort + 1;
  int* s_consumed = s_abort + 2;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nloc = blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const tc::Guard guard{s_abort, a.status, a.wait_ns};

  if (tid == 0) {
    for (int i = 0; i < kUpdStages; ++i) {
      tc::mbar_init(full + i, 1);
      tc::mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(acc_full + i, 1);
      tc::mbar_init(acc_empty + i, 128);
    }
    tc::mbar_init(fin, 1);
    *s_abort = 0;
    *s_issued = 0;
    *s_consumed = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, NCOL);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;

  if (warp == 0 && lane == 0) {
    int k = 0;
    for (int li = 0; li < nloc && !*s_abort; ++li) {
      const int64_t tile = blockIdx.x + (int64_t)li * gridDim.x;
      for (int G = a.G0; G < a.G1; ++G, ++k) {
        const int stage = k % kUpdStages, u = k / kUpdStages;
        if (u >= 1 && !tc::mbar_wait(empty + stage, (u - 1) & 1, guard, kErrWaitProducer)) goto produced;
        tc::mbar_expect_tx(full + stage, STAGE);
        uint8_t* dst = smem + stage * STAGE;
        for (int mg = 0; mg < 16; ++mg)
          tc::bulk_g2s(dst + mg * kStrip, a.q + ((size_t)(G * 16 + mg) * a.n_oct + tile * (kChunk / 8)) * 128,
                       kStrip, full + stage);
        tc::bulk_g2s(dst + kAStage, a.hs + (size_t)G * NP * 16, HB, full + stage);
      }
    }
  produced:
    *s_issued = k;
  } else if (warp == 1 && lane == 0) {
    int k = 0;
    bool ok = true;
    for (int li = 0; li < nloc && ok; ++li) {
      const int buf = li % NBUF;
      if (li >= NBUF && !tc::mbar_wait(acc_empty + buf, ((li / NBUF) - 1) & 1, guard, kErrWaitMma)) break;
      tc::fence_after_sync();
      for (int G = a.G0; G < a.G1; ++G, ++k) {
        const int stage = k % kUpdStages, u = k / kUpdStages;
        if (!tc::mbar_wait(full + stage, u & 1, guard, kErrWaitMma)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t base = tc::smem_u32(smem + stage * STAGE);
        // B: K-major, column halves (c/8) 128 B apart along K, j blocks 256 B apart along N
        const uint64_t bd = tc::smem_desc(base + kAStage, 128, 256);
#pragma unroll
        for (int s = 0; s < kDig; ++s) {
          // A: MN-major, strips 2s (columns 0-7) and 2s+1 (8-15) one strip apart
          // along K, row octets 128 B apart along M
          const uint64_t ad = tc::smem_desc(base + 2 * s * kStrip, kStrip, 128);
          tc::mma_bf16(tmem + (uint32_t)(buf * kDig * NP + s * NP), ad, bd, IDESC, G != a.G0);
        }
        tc::mma_commit(empty + stage);
      }
      if (!ok) break;
      tc::mma_commit(acc_full + buf);
    }
    *s_consumed = k;
    tc::mma_commit(fin);
  } else if (warp >= 2) {
    const int q4 = warp & 3;
    const int m = q4 * 32 + lane;
    double hsc[NJ];
    uint32_t wm[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      hsc[j] = j < a.r ? pow2i(a.hexp[j] - 28) : 0.0;
      wm[j] = 0u;
    }
    for (int li = 0; li < nloc; ++li) {
      const int buf = li % NBUF;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(acc_full + buf, (li / NBUF) & 1, guard, kErrWaitEpilogue))) break;
      tc::fence_after_sync();
      int S[NJ][9];
#pragma unroll
      for (int j = 0; j < NJ; ++j)
#pragma unroll
        for (int d = 0; d < 9; ++d) S[j][d] = 0;
#pragma unroll
      for (int s = 0; s < kDig; ++s) {
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * kDig * NP + s * NP);
        uint32_t v[NP];
        if constexpr (NP == 16) {
          tc::tmem_ld16(taddr, v);
        } else {
#pragma unroll
          for (int c = 0; c < NP / 32; ++c) {
            uint32_t h[32];
            tc::tmem_ld32(taddr + 32 * c, h);
#pragma unroll
            for (int x = 0; x < 32; ++x) v[32 * c + x] = h[x];
          }
        }
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < NP / 8; ++j)
#pragma unroll
          for (int t = 0; t < kDig; ++t)
            if (s + t <= 8) S[j][s + t] += exact_int(v[j * 8 + t]);
      }
      tc::fence_before_sync();
      tc::mbar_arrive(acc_empty + buf);
      const int64_t i = (blockIdx.x + (int64_t)li * gridDim.x) * kChunk + m;
      if (i < a.n) {
#pragma unroll
        for (int j = 0; j < NP / 8; ++j) {
          if (j < a.r) {
            const long long P0 = ((long long)S[j][0] << 16) + ((long long)S[j][1] << 8) + S[j][2];
            const long long P1 = ((long long)S[j][3] << 16) + ((long long)S[j][4] << 8) + S[j][5];
            const long long P2 = ((long long)S[j][6] << 16) + ((long long)S[j][7] << 8) + S[j][8];
            const double val =
                ((small_ll_to_double(P2) * 5.9604644775390625e-08 + small_ll_to_double(P1)) * 5.9604644775390625e-08 +
                 small_ll_to_double(P0)) *
                hsc[j];
            const double w = a.keep ? a.W[i * a.ldw + j] - val : -val;
            a.W[i * a.ldw + j] = w;
            wm[j] = max(wm[j], abs_hiword(w));
          }
        }
      }
    }
    if (a.wmax_out) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const uint32_t w = __reduce_max_sync(0xffffffffu, wm[j]);
        if (lane == 0 && j < a.r && w) atomicMax(a.wmax_out + j, w);
      }
    }
  }

  __syncthreads();
  if (tid == 0) {
    tc::mbar_wait_drain(fin, 0);
    for (int k = *s_consumed; k < *s_issued; ++k)
      tc::mbar_wait_drain(full + (k % kUpdStages), (k / kUpdStages) & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, NCOL);
  }
}

// ---------------------------------------------------------------------------
constexpr int kProbeA = 36 * 1024, kProbeB = 20 * 1024;
// One MMA of a 128 x 16 A tile and an NP x 16 B tile given as shared-memory
// images with explicit descriptor strides (the layout check of the C ABI).
__global__ void tc_probe_kernel(const uint4* a_img, int a_words, const uint4* b_img, int b_words, int np,
                                int a_mn_major, uint32_t a_lbo, uint32_t a_sbo, uint32_t b_lbo, uint32_t b_sbo,
                                float* out, int* status, uint64_t wait_ns) {
  constexpr int ABYTES = kProbeA, BBYTES = kProbeB;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint4* sa = reinterpret_cast<uint4*>(smem);
  uint4* sb = reinterpret_cast<uint4*>(smem + ABYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + ABYTES + BBYTES);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);
  int* s_abort = reinterpret_cast<int*>(s_tmem + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < ABYTES / 16; i += blockDim.x) sa[i] = i < a_words ? a_img[i] : make_uint4(0, 0, 0, 0);
  for (int i = tid; i < BBYTES / 16; i += blockDim.x) sb[i] = i < b_words ? b_img[i] : make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async_smem();
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    *s_abort = 0;
    tc::fence_mbar_init();
  }
  const uint32_t ncols = np < 32 ? 32 : np;
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, np, a_mn_major, 0);
    tc::mma_bf16(tmem, tc::smem_desc(tc::smem_u32(sa), a_lbo, a_sbo), tc::smem_desc(tc::smem_u32(sb), b_lbo, b_sbo),
                 idesc, 0);
    tc::mma_commit(bar);
  }
  const tc::Guard guard{s_abort, status, wait_ns};
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(bar, 0, guard, kErrWaitEpilogue));
  tc::fence_after_sync();
  if (ok) {
    for (int c = 0; c < (np + 31) / 32; ++c) {
      uint32_t v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * c, v);
      tc::tmem_ld_wait();
      for (int x = 0; x < 32 && 32 * c + x < np; ++x)
        out[(warp * 32 + lane) * np + 32 * c + x] = __uint_as_float(v[x]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, ncols);
  }
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    FLZ_CUDA(cudaGetDevice(&dev));
    FLZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

template <class K>
void allow_smem(K kernel, size_t bytes) {
  FLZ_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

constexpr size_t kBarBytes = 256;
size_t dot_smem(int np) { return (size_t)dot_stages(np) * kAStage + 2 * (size_t)np * kRange * 2 + kBarBytes; }
size_t upd_smem(int np) { return (size_t)kUpdStages * (kAStage + np * 32) + kUpdPad + kBarBytes; }

// N of an MMA holding r columns x 8 digits: a multiple of 16 (M = 128)
int padded_np(int r) { return r <= 2 ? 16 : r <= 4 ? 32 : r <= 8 ? 64 : 128; }

template <int NP>
void launch_dot(TcBasis& B, int K, const double* W, int r, int ldw, const uint32_t* wmax, double* C, int ldc,
                cudaStream_t st) {
  constexpr int GPC = 128 / NP;
  const int Gtot = (K + 15) / 16;
  const int GS = (Gtot + GPC - 1) / GPC;
  const int nR = (int)(B.n_pad / kRange);
  const int minRS = (nR + 255) / 256;  // <= 256 ranges per CTA keeps the int32 sums exact
  const int sms = num_sms();
  const int waves = std::max(1, (minRS * GS + sms - 1) / sms);
  int RS = std::max(minRS, (waves * sms) / GS);
  RS = std::max(1, std::min(RS, nR));
  const size_t wbytes = (size_t)B.n_pad * NP * 2;
  if (B.wd.count < wbytes) B.wd.reserve(wbytes);
  static bool attr = false;
  if (!attr) {
    allow_smem(tc_dot_kernel<NP>, dot_smem(NP));
    attr = true;
  }
  const int64_t tasks = B.n_oct * (NP / 8);
  w_digits_kernel<<<(unsigned)((tasks + 255) / 256), 256, 0, st>>>(W, B.n, r, ldw, wmax, NP, B.n_oct, B.wd.p);
  FLZ_LAUNCH_CHECK();
  DotArgs a{B.q.p, B.wd.p, B.n_oct, Gtot, nR, RS, B.acc.p, B.status.p, wait_limit_ns()};
  tc_dot_kernel<NP><<<dim3(GS, RS), 192, dot_smem(NP), st>>>(a);
  FLZ_LAUNCH_CHECK();
  tc_dot_reduce_kernel<NP><<<Gtot, 16 * r, 0, st>>>(B.acc.p, K, r, wmax, C, ldc);
  FLZ_LAUNCH_CHECK();
}

// keep = 1: W -= Q[:, :K] H; keep = 0: W = -Q[:, :K] H in the first window, later windows subtract
template <int NP>
void launch_update(TcBasis& B, int K, double* W, int r, int ldw, int keep, uint32_t* wmax_out, cudaStream_t st) {
  const int Gtot = (K + 15) / 16;
  const int ntiles = (int)(B.n_pad / kChunk);
  const int grid = std::min(ntiles, num_sms());
  static bool attr = false;
  if (!attr) {
    allow_smem(tc_update_kernel<NP>, upd_smem(NP));
    attr = true;
  }
  for (int G0 = 0; G0 < Gtot; G0 += kWindowGroups) {
    const int G1 = std::min(Gtot, G0 + kWindowGroups);
    UpdArgs a{B.q.p, B.n_oct, B.n, ntiles, G0, G1, B.hs.p, B.hexp.p, W, r, ldw, keep || G0 > 0 ? 1 : 0,
              G1 == Gtot ? wmax_out : nullptr, B.status.p, wait_limit_ns()};
    tc_update_kernel<NP><<<grid, 192, upd_smem(NP), st>>>(a);
    FLZ_LAUNCH_CHECK();
  }
}

}  // namespace

bool TcBasis::supported(int r) { return r >= 1 && r <= 16; }

void TcBasis::release() {
  q.release();
  acc.release();
  wd.release();
  hs.release();
  hexp.release();
  wmax.release();
  status.release();
  if (status_host) cudaFreeHost(status_host);
  status_host = nullptr;
  n = n_pad = n_oct = 0;
  groups_cap = 0;
}

size_t TcBasis::bytes_for(int64_t n, int64_t kcap) {
  const int64_t n_pad = (n + kRange - 1) / kRange * kRange;
  const int64_t groups = (kcap + 15) / 16;
  return (size_t)groups * 16 * (size_t)n_pad * 16;
}

void TcBasis::reserve(int64_t n_, int64_t kcap) {
  const int64_t n_pad_ = (n_ + kRange - 1) / kRange * kRange;
  const int groups = (int)((kcap + 15) / 16);
  if (q.p && n == n_ && groups <= groups_cap) return;
  release();
  n = n_;
  n_pad = n_pad_;
  n_oct = n_pad / 8;
  groups_cap = groups;
  const size_t bytes = bytes_for(n_, kcap);
  q.reserve(bytes);
  // digits outside the written columns and rows must be finite (zero)
  FLZ_CUDA(cudaMemset(q.p, 0, bytes));
  hs.reserve((size_t)groups_cap * 64 * 16 + 64);  // update N <= 64
  acc.reserve((size_t)groups_cap * 128 * 128);    // 128 x N sums per group, N <= 128
  FLZ_CUDA(cudaMemset(acc.p, 0, sizeof(unsigned long long) * acc.count));
  hexp.reserve(16);
  wmax.reserve(32);
  status.reserve(1);
  FLZ_CUDA(cudaMemset(status.p, 0, sizeof(int)));
  FLZ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&status_host), sizeof(int)));
  *status_host = 0;
}

void TcBasis::grow(int64_t kcap, cudaStream_t st) {
  const int groups = (int)((kcap + 15) / 16);
  if (groups <= groups_cap) return;
  const int ng = std::max(groups, 2 * groups_cap);
  // groups are contiguous, group-major: the written ones are a prefix
  const size_t old_bytes = (size_t)groups_cap * 16 * (size_t)n_pad * 16;
  const size_t bytes = (size_t)ng * 16 * (size_t)n_pad * 16;
  DevBuf<uint8_t> nq;
  nq.reserve(bytes);
  FLZ_CUDA(cudaMemcpyAsync(nq.p, q.p, old_bytes, cudaMemcpyDeviceToDevice, st));
  FLZ_CUDA(cudaMemsetAsync(nq.p + old_bytes, 0, bytes - old_bytes, st));
  FLZ_CUDA(cudaStreamSynchronize(st));  // the old copy is freed on return
  std::swap(q.p, nq.p);
  std::swap(q.count, nq.count);
  hs.reserve((size_t)ng * 64 * 16 + 64);
  acc.reserve((size_t)ng * 128 * 128);  // zero between projections
  FLZ_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * acc.count, st));
  groups_cap = ng;
}

void TcBasis::reshape(int64_t n_, int64_t kcap, cudaStream_t st) {
  const int64_t n_pad_ = (n_ + kRange - 1) / kRange * kRange;
  const int groups = (int)((kcap + 15) / 16);
  const size_t bytes = (size_t)groups * 16 * (size_t)n_pad_ * 16;
  if (!q.p || q.count < bytes || acc.count < (size_t)groups * 128 * 128 ||
      hs.count < (size_t)groups * 64 * 16 + 64 || !status.p) {
    release();
    reserve(n_, kcap);
    return;
  }
  n = n_;
  n_pad = n_pad_;
  n_oct = n_pad / 8;
  groups_cap = groups;
  FLZ_CUDA(cudaMemsetAsync(q.p, 0, bytes, st));  // digits outside the written columns and rows must be zero
}

void TcBasis::append(double* X, int r, int col0, cudaStream_t st) {
  if (col0 + r > groups_cap * 16) fail(FLZ_ERR_CAPACITY, "digit basis holds %d columns", groups_cap * 16);
  const int64_t work = n_oct * r;
  const int threads = 256;
  basis_digits_kernel<<<(unsigned)((work + threads - 1) / threads), threads, 0, st>>>(X, n, r, col0, q.p, n_oct);
  FLZ_LAUNCH_CHECK();
}

void TcBasis::project(int K, const double* W, int r, int ldw, const uint32_t* wmax_in, double* C, int ldc,
                      cudaStream_t st) {
  switch (padded_np(r)) {
    case 16: launch_dot<16>(*this, K, W, r, ldw, wmax_in, C, ldc, st); break;
    case 32: launch_dot<32>(*this, K, W, r, ldw, wmax_in, C, ldc, st); break;
    case 64: launch_dot<64>(*this, K, W, r, ldw, wmax_in, C, ldc, st); break;
    default: launch_dot<128>(*this, K, W, r, ldw, wmax_in, C, ldc, st); break;
  }
}

namespace {
// W[:, c0:c0+w] op= Q H[:, c0:c0+w] for w <= 8 columns (one digit set of H)
void update_columns(TcBasis& B, int K, const double* C, int ldc, int w, double* W, int ldw, int keep, int sign,
                    uint32_t* wmax_out, cudaStream_t st) {
  const int np = std::min(padded_np(w), 64);
  const int Gtot = (K + 15) / 16;
  tc_hdigits_kernel<<<1, 256, 0, st>>>(C, ldc, K, w, Gtot, np, B.hs.p, B.hexp.p, sign);
  FLZ_LAUNCH_CHECK();
  switch (np) {
    case 16: launch_update<16>(B, K, W, w, ldw, keep, wmax_out, st); break;
    case 32: launch_update<32>(B, K, W, w, ldw, keep, wmax_out, st); break;
    default: launch_update<64>(B, K, W, w, ldw, keep, wmax_out, st); break;
  }
}
}  // namespace

void TcBasis::subtract(int K, const double* C, int ldc, double* W, int r, int ldw, uint32_t* wmax_out,
                       cudaStream_t st) {
  for (int c0 = 0; c0 < r; c0 += 8)  // at most 8 columns (N = 64) per pass over the digits
    update_columns(*this, K, C + c0, ldc, std::min(8, r - c0), W + c0, ldw, 1, 1,
                   wmax_out ? wmax_out + c0 : nullptr, st);
}

void TcBasis::multiply(int K, const double* C, int ldc, int s, double* X, int ldx, cudaStream_t st) {
  // digits of -C: the first window writes -Q(-C), later windows subtract Q(-C)
  for (int c0 = 0; c0 < s; c0 += 8)
    update_columns(*this, K, C + c0, ldc, std::min(8, s - c0), X + c0, ldx, 0, -1, nullptr, st);
}

void TcBasis::column_max(const double* W, int r, int ldw, uint32_t* out, cudaStream_t st) {
  FLZ_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t) * 16, st));
  colmax_kernel<<<2 * num_sms(), 256, 0, st>>>(W, n, r, ldw, out);
  FLZ_LAUNCH_CHECK();
}

void TcBasis::cgs2(int K, double* W, int r, double* C, double* C2, cudaStream_t st) {
  uint32_t* m0 = wmax.p;
  uint32_t* m1 = wmax.p + 16;
  column_max(W, r, r, m0, st);
  project(K, W, r, r, m0, C, r, st);
  FLZ_CUDA(cudaMemsetAsync(m1, 0, sizeof(uint32_t) * 16, st));
  subtract(K, C, r, W, r, r, m1, st);
  project(K, W, r, r, m1, C2, r, st);
  subtract(K, C2, r, W, r, r, nullptr, st);
  FLZ_CUDA(cudaMemcpyAsync(status_host, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
}

void TcBasis::check_status() {
  if (status_host && *status_host) {
    const int code = *status_host;
    // reported once: the next call starts from a clear status
    *status_host = 0;
    cudaMemset(status.p, 0, sizeof(int));
    fail(FLZ_ERR_TIMEOUT, "tensor-core reorthogonalization: a wait expired (role %d)", code);
  }
}

int tc_probe(const uint16_t* a_img, size_t a_bytes, const uint16_t* b_img, size_t b_bytes, int np, int a_mn_major,
             uint32_t a_lbo, uint32_t a_sbo, uint32_t b_lbo, uint32_t b_sbo, float* out_host) {
  if (np != 16 && np != 32 && np != 64 && np != 128) fail(FLZ_ERR_INVALID_ARG, "np must be 16, 32, 64 or 128");
  if (a_bytes % 16 || b_bytes % 16 || a_bytes > (size_t)kProbeA || b_bytes > (size_t)kProbeB)
    fail(FLZ_ERR_INVALID_ARG, "images must be multiples of 16 bytes, at most %d and %d bytes", kProbeA, kProbeB);
  for (uint32_t x : {a_lbo, a_sbo, b_lbo, b_sbo})
    if (x % 16 || x > 8192) fail(FLZ_ERR_INVALID_ARG, "descriptor strides must be multiples of 16 up to 8192");
  // every fetch stays inside the staged images under either reading of the two stride fields
  const uint64_t ga = 15, gb = (uint64_t)np / 8 - 1;
  if (ga * a_sbo + a_lbo + 128 > kProbeA || ga * a_lbo + a_sbo + 128 > kProbeA ||
      gb * b_sbo + b_lbo + 128 > kProbeB || gb * b_lbo + b_sbo + 128 > kProbeB)
    fail(FLZ_ERR_INVALID_ARG, "descriptor strides reach past the staged images");
  DevBuf<uint4> da, db;
  DevBuf<float> dout;
  DevBuf<int> dst;
  const int aw = (int)(a_bytes / 16), bw = (int)(b_bytes / 16);
  da.reserve(std::max(aw, 1));
  db.reserve(std::max(bw, 1));
  dout.reserve((size_t)128 * np);
  dst.reserve(1);
  FLZ_CUDA(cudaMemcpy(da.p, a_img, a_bytes, cudaMemcpyHostToDevice));
  FLZ_CUDA(cudaMemcpy(db.p, b_img, b_bytes, cudaMemcpyHostToDevice));
  FLZ_CUDA(cudaMemset(dout.p, 0, sizeof(float) * 128 * np));
  FLZ_CUDA(cudaMemset(dst.p, 0, sizeof(int)));
  const size_t smem = kProbeA + kProbeB + 64;
  allow_smem(tc_probe_kernel, smem);
  tc_probe_kernel<<<1, 128, smem>>>(da.p, aw, db.p, bw, np, a_mn_major, a_lbo, a_sbo, b_lbo, b_sbo, dout.p, dst.p,
                                    wait_limit_ns());
  FLZ_LAUNCH_CHECK();
  FLZ_CUDA(cudaDeviceSynchronize());
  int status = 0;
  FLZ_CUDA(cudaMemcpy(&status, dst.p, sizeof(int), cudaMemcpyDeviceToHost));
  FLZ_CUDA(cudaMemcpy(out_host, dout.p, sizeof(float) * 128 * np, cudaMemcpyDeviceToHost));
  return status;
}

}  // namespace flz
