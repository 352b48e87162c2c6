// Device building blocks of the phase-tracking hot path (arxiv 1906.10598).
//
// Model (Sec. 2.2 Eq. 2-2-2, c5 = 0) in cycles:
//   m(t) = A cos(2 pi p(t)),  p(t) = phi0/(2 pi) + f0 t + f1 t^2/2 + f2 t^3/6,
// objective (Eq. 2-2-4): SSE = sum_i (s_i - m(t_i))^2, t_i = t0 + i h, h = 1/fs.
//
// Default-tier phase pipeline (FP64-accurate, FP32 arithmetic in the sample loop):
//   1. per candidate, FP64: the phase as a polynomial in the sample index,
//        p(t0 + i h) = E0 + E1 i + E2 i^2 + E3 i^3,
//      each coefficient reduced mod 1 exactly into a 128-bit binary fraction;
//   2. per (candidate, 256-sample tile starting at i0), integer arithmetic mod
//      2^128 re-expands the polynomial at i0 (exact):
//        p(i0 + k) = P + D1 k + D2 k^2 + D3 k^3  (mod 1);
//   3. per sample, the linear part walks in 32-bit fixed point (wrapping is
//      the reduction mod one cycle), the small k^2/k^3 terms are FP32, and
//      the SFU cosine takes the phase in radians in [-pi, pi) plus the small terms.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace pt {

typedef unsigned __int128 u128;

constexpr int D = 5;             // (A, phi0, f0, f1, f2)
// The full model: Eq. 2-2-2 with the amplitude slope c5 (A1) and the phase of
// Eq. 2-2-1 to order n = 4 (Sec. 3.2, arcs near perigee),
//   m(t) = (A + A1 t) cos(2 pi p(t)),  p(t) = ... + f3 t^4 / 24,
// parameters (A, phi0, f0, f1, f2, A1, f3).
constexpr int DF = 7;
constexpr int MODEL_CUBIC = 0;
constexpr int MODEL_FULL = 1;
__host__ __device__ constexpr int model_dim(int model) { return model == MODEL_FULL ? DF : D; }
constexpr int M = 8;             // samples per lane per tile
constexpr int L = 32 * M;        // samples per tile
constexpr int NP_MAX = 128;      // largest population / candidate batch per CTA
// Each candidate's word of the DE exchange ring sits on its own 128-byte line,
// so the arrivals and polls of different candidates go to different L2 lines.
constexpr int RING_STRIDE = 16;
// A ring word's low byte counts the group's arrivals: at most 255 CTAs per group.
constexpr int DE_GROUP_MAX = 255;
// Generations the DE exchange ring holds (see de_block: slot g + 2 is cleared
// during generation g's wait).
constexpr int RING_SLOTS = 4;

constexpr double TWO_PI = 2.0 * 3.14159265358979323846;
constexpr double INV_TWO_PI = 0.15915494309189533577;
// 2 pi / 2^32 and 2 pi / 2^64 as FP32 scale factors of fixed-point phases
constexpr float TWO_PI_2M32 = 1.46291807926715968e-09f;
constexpr float TWO_PI_2M64 = 3.40612158008655460e-19f;

// Status written by a kernel into its error word (0 = OK).
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = 1;   // a bounded wait expired
constexpr int DEV_LAYOUT = 2;    // a CTA's tiles exceed the resident layout its kernel was compiled for

// Per-block constants shared by all kernels.
struct BlockArgs {
  const void* samples;   // device; zero-padded to a multiple of L samples
  int64_t n;             // valid samples
  int64_t ntiles;        // ceil(n / L)
  int dtype;             // PT_I8 .. PT_F64
  int esize;             // bytes per stored sample
  double scale;          // physical = scale * stored
  double smax;           // max |physical sample|
  float smax_f;          // smax rounded to FP32 (sets the SSE fixed-point scale)
  double t0, h;          // t_i = t0 + i h
  double t0sq_2, t0cu_6; // t0^2/2, t0^3/6
  double h2_2, h3_6;     // h^2/2, h^3/6
  double t0qu_24, h4_24; // t0^4/24, h^4/24 (full model)
  double quartic_k3, quartic_k4;  // 2 pi (M/2)^3 and 2 pi ((M/2)^4 + 4 (n + 2 L) (M/2)^3), see quartic_needed
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Twelve words for individual `ind` at generation `gen`: counters (g, ind, gen, block) for g = 0, 1, 2.
__device__ __forceinline__ void de_draw12(uint2 key, uint32_t block_id, uint32_t gen, uint32_t ind, uint32_t w[12]) {
#pragma unroll
  for (uint32_t g = 0; g < 3; ++g) {
    uint4 r = philox4x32_10(make_uint4(g, ind, gen, block_id), key);
    w[4 * g + 0] = r.x;
    w[4 * g + 1] = r.y;
    w[4 * g + 2] = r.z;
    w[4 * g + 3] = r.w;
  }
}

// Integer in [0, k) from one word (Lemire multiply-shift).
__device__ __forceinline__ uint32_t lemire(uint32_t w, uint32_t k) {
  return (uint32_t)(((uint64_t)w * (uint64_t)k) >> 32);
}

// Uniform double in [0, 1) from 27 + 26 random bits.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return __dmul_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)), 1.0 / 9007199254740992.0);
}

// DE controls shared by the kernels.
// Mutation strategies (Table 3-1-1 names them by number: "3" for the
// chi-square, "6" for the correlation objective, Sec. 3.1.2; read in the
// order of Price, Storn & Lampinen 2006, which the paper cites):
//   DE_RAND1_BIN     v = x_r1 + F (x_r2 - x_r3), binomial crossover (default);
//   DE_BEST1_JITTER  v_j = x_best,j + F_j (x_r2,j - x_r3,j), F_j = F + 1e-4 U_j,
//                    binomial crossover, x_best the previous generation's
//                    lowest-index minimum;
//   DE_EITHER_OR     with probability 1/2 the rand/1 mutant, otherwise
//                    x_r1 + K ((x_r2 + x_r3) - 2 x_r1), K = (F + 1)/2; no crossover.
constexpr int DE_RAND1_BIN = 0;
constexpr int DE_BEST1_JITTER = 3;
constexpr int DE_EITHER_OR = 6;

struct DeControls {
  double lo[DF], hi[DF];  // the first model_dim(model) entries are used
  double F;
  double K;          // (F + 1) / 2, for DE_EITHER_OR
  uint32_t cr_thr;   // crossover if word < cr_thr
  int cr_all;        // CR >= 1
  int periodic;      // phi0 range spans the full circle
  int strategy;      // DE_*
  uint2 key;         // Philox key (seed lo, seed hi)
  uint32_t block_id;
};

// Generation-0 individual: uniform inside the bounds; component j from words
// 2j, 2j+1 (words 12, 13 from counter group 3 for the full model's last one).
template <int DIM = D>
__device__ __forceinline__ void de_init(const DeControls& dc, int i, double* xi) {
  uint32_t w[14];
  de_draw12(dc.key, dc.block_id, 0u, (uint32_t)i, w);
  if (DIM > 6) {
    const uint4 g3 = philox4x32_10(make_uint4(3u, (uint32_t)i, 0u, dc.block_id), dc.key);
    w[12] = g3.x;
    w[13] = g3.y;
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j)
    xi[j] = __dadd_rn(dc.lo[j], __dmul_rn(u53(w[2 * j], w[2 * j + 1]), __dsub_rn(dc.hi[j], dc.lo[j])));
}

// Order-preserving integer key of a finite double: a < b  <=>  key(a) < key(b).
// Comparisons in the DE run on the integer pipes (B300's FP64 pipe is 1/64 rate).
__device__ __forceinline__ long long dkey(double a) {
  const long long b = __double_as_longlong(a);
  return b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b);
}

// Random draws of individual i at generation gen >= 1 (selection-independent):
// r1, r2, r3 packed in bytes 0..2 (distinct, != i), crossover mask in `take`
// (bit j set = component j comes from the mutant).
// DE_EITHER_OR marks a three-point trial in bit 24 of rpack and takes every
// component; DE_BEST1_JITTER also writes the DIM jitter words of the trial
// (words 9..11, then words 0..DIM-4 of a fourth counter group) to jit[0..DIM-1].
template <int STRAT, int DIM = D>
__device__ __forceinline__ void de_draws(const DeControls& dc, int np, int i, uint32_t gen, uint32_t* rpack,
                                         uint32_t* take, uint32_t* jit) {
  uint32_t w[12];
  de_draw12(dc.key, dc.block_id, gen, (uint32_t)i, w);
  if (STRAT == DE_BEST1_JITTER) {
    const uint4 g3 = philox4x32_10(make_uint4(3u, (uint32_t)i, gen, dc.block_id), dc.key);
    jit[0] = w[9];
    jit[1] = w[10];
    jit[2] = w[11];
    jit[3] = g3.x;
    jit[4] = g3.y;
    if (DIM > 5) {
      jit[5] = g3.z;
      jit[6] = g3.w;
    }
  }
  // three distinct indices != i, by index shifting over the sorted exclusions
  uint32_t excl[4];
  uint32_t r[3];
  int nex = 1;
  excl[0] = (uint32_t)i;
  for (int d = 0; d < 3; ++d) {
    uint32_t v = lemire(w[d], (uint32_t)np - 1u - (uint32_t)d);
    for (int e = 0; e < nex; ++e)  // excl is sorted ascending
      if (v >= excl[e]) v++;
    r[d] = v;
    int pos = nex;  // insertion keeps excl sorted
    while (pos > 0 && excl[pos - 1] > v) {
      excl[pos] = excl[pos - 1];
      --pos;
    }
    excl[pos] = v;
    nex++;
  }
  const uint32_t jrand = lemire(w[3], (uint32_t)DIM);
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < DIM; ++j)
    if ((uint32_t)j == jrand || dc.cr_all || w[4 + j] < dc.cr_thr) m |= 1u << j;
  *rpack = r[0] | (r[1] << 8) | (r[2] << 16);
  *take = m;
  if (STRAT == DE_EITHER_OR) {
    *take = (1u << DIM) - 1u;
    if (w[9] >= 0x80000000u) *rpack |= 1u << 24;
  }
}

// x * 0.5, exactly as the FP64 multiply would round it: when x is normal and
// x/2 is too, halving only decrements the exponent field (integer pipe);
// otherwise multiply.
__device__ __forceinline__ double half_exact(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  return (e > 1 && e < 0x7FF) ? __longlong_as_double(b - (1ll << 52)) : __dmul_rn(x, 0.5);
}

// Component j of the DE trial of individual i from population x (np x DIM). FP64 operations use _rn intrinsics so no contraction changes a
// rounding: the value is bit-identical to a plain IEEE evaluation.
// STRAT is the DE_* strategy (a template parameter, so each strategy's loop
// holds only its own FP64 operations); `best` (the previous generation's
// lowest-index minimum) and jit (the trial's five jitter words) are used by
// DE_BEST1_JITTER only.
template <int STRAT, int DIM = D>
__device__ __forceinline__ double de_component(const DeControls& dc, const double* x, int i, int j, uint32_t rpack,
                                               uint32_t take, int best, const uint32_t* jit) {
  const double parent = x[i * DIM + j];
  if (!((take >> j) & 1u)) return parent;
  const int r0 = rpack & 0xff, r1 = (rpack >> 8) & 0xff, r2 = (rpack >> 16) & 0xff;
  double v;
  if (STRAT == DE_BEST1_JITTER) {
    const double Fj = __dadd_rn(dc.F, __dmul_rn(1e-4, (double)jit[j] * (1.0 / 4294967296.0)));
    v = __dadd_rn(x[best * DIM + j], __dmul_rn(Fj, __dsub_rn(x[r1 * DIM + j], x[r2 * DIM + j])));
  } else if (STRAT == DE_EITHER_OR) {
    const double a = x[r0 * DIM + j], b = x[r1 * DIM + j], c = x[r2 * DIM + j];
    if (rpack >> 24) v = __dadd_rn(a, __dmul_rn(dc.K, __dsub_rn(__dadd_rn(b, c), 2.0 * a)));
    else v = __dadd_rn(a, __dmul_rn(dc.F, __dsub_rn(b, c)));
  } else {
    v = __dadd_rn(x[r0 * DIM + j], __dmul_rn(dc.F, __dsub_rn(x[r1 * DIM + j], x[r2 * DIM + j])));
  }
  if (j == 1 && dc.periodic) {
    const double d = __dsub_rn(v, dc.lo[j]);
    // k = floor(fl(d / 2pi)) without dividing: for d in [-4pi, 5pi) the
    // quotient crosses -1, 0, 1, 2 exactly where d crosses the exact doubles
    // -2pi, 0, 2pi, 4pi (the quotient's rounding threshold lies within half
    // an ulp of d of each), so comparing d with them gives the same k as the
    // rounded division; outside that range, divide.
    const long long kd = dkey(d);
    double k;
    if (kd >= dkey(-2.0 * TWO_PI) && kd < dkey(2.5 * TWO_PI)) {
      k = kd >= dkey(2.0 * TWO_PI) ? 2.0
          : kd >= dkey(TWO_PI)     ? 1.0
          : kd >= dkey(0.0)        ? 0.0
          : kd >= dkey(-TWO_PI)    ? -1.0
                                   : -2.0;
    } else {
      k = floor(__ddiv_rn(d, TWO_PI));
    }
    if (k != 0.0) v = __dsub_rn(v, __dmul_rn(k, TWO_PI));
  } else if (dkey(v) < dkey(dc.lo[j])) {
    v = half_exact(__dadd_rn(dc.lo[j], parent));
  } else if (dkey(v) > dkey(dc.hi[j])) {
    v = half_exact(__dadd_rn(dc.hi[j], parent));
  }
  return v;
}

// ---------------------------------------------------------------------------
// Fixed-point phase polynomial.

// frac(x) as a 128-bit binary fraction (x * 2^128 mod 2^128), exact for any
// finite double (bits below 2^-128 are truncated).
__device__ __forceinline__ u128 frac128(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) return 0;
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1075 + 128;  // x * 2^128 = mant * 2^sh
  u128 r;
  if (sh >= 128) r = 0;
  else if (sh >= 0) r = ((u128)mant) << sh;
  else if (sh > -64) r = (u128)(mant >> (-sh));
  else r = 0;
  if (b >> 63) r = (u128)0 - r;
  return r;
}

struct Poly {
  u128 e[4];  // E0..E3 as fractions of a cycle
};

// Coefficient E_k (k = 0..3) of candidate th = (A, phi0, f0, f1, f2) for the
// block's time base, reduced mod 1 into a 128-bit fraction:
//   E3 = f2 h^3/6,  E2 = (f1 + f2 t0) h^2/2,  E1 = (f0 + f1 t0 + f2 t0^2/2) h,
//   E0 = phi0/(2 pi) + f0 t0 + f1 t0^2/2 + f2 t0^3/6.
__device__ __forceinline__ double poly_coef(const double* th, const BlockArgs& b, int k) {
  const double phi0 = th[1], f0 = th[2], f1 = th[3], f2 = th[4];
  if (k == 3) return f2 * b.h3_6;
  if (k == 2) return fma(f2, b.t0, f1) * b.h2_2;
  if (k == 1) return fma(f2, b.t0sq_2, fma(f1, b.t0, f0)) * b.h;
  return fma(f2, b.t0cu_6, fma(f1, b.t0sq_2, fma(f0, b.t0, phi0 * INV_TWO_PI)));
}
__device__ __forceinline__ u128 poly_term(const double* th, const BlockArgs& b, int k) {
  return frac128(poly_coef(th, b, k));
}

// Inside a lane's run of M consecutive samples k = kc + m' of a tile (kc =
// k0 + M/2, m' in [-M/2, M/2)), the cubic term E3 k^3 may be folded into the
// quadratic one as k^2 (E2 + E3 kc), with an error |E3| k^2 |m'| <=
// |E3| (L - 1)^2 M / 2. A candidate keeps the exact cubic when that bound, in
// radians, exceeds 2^-24 (below the FP32 rounding of the phase argument
// itself), i.e. when |E3| (cycles per sample^3) exceeds CUBIC_FOLD_MAX.
constexpr double CUBIC_FOLD_MAX = 5.9604644775390625e-08 / (6.283185307179586 * (L - 1) * (L - 1) * 0.5 * M);
__device__ __forceinline__ bool cubic_needed(double E3) {
  return (__double_as_longlong(E3) & 0x7fffffffffffffffll) > __double_as_longlong(CUBIC_FOLD_MAX);
}

// x * y mod 2^128 for a 64-bit y.
__device__ __forceinline__ u128 mul_u128_u64(u128 x, uint64_t y) {
  const uint64_t xl = (uint64_t)x, xh = (uint64_t)(x >> 64);
  const uint64_t lo = xl * y, hi = __umul64hi(xl, y) + xh * y;
  return ((u128)hi << 64) | lo;
}

// A signed 64-bit integer as FP32 (two 32-bit conversions, relative error
// below 2^-23), avoiding the slow 64-bit conversion path.
__device__ __forceinline__ float i64_to_f32(long long v) {
  const bool neg = v < 0;
  const unsigned long long a = neg ? (0ull - (unsigned long long)v) : (unsigned long long)v;
  const float f = fmaf((float)(uint32_t)(a >> 32), 4294967296.0f, (float)(uint32_t)a);
  return neg ? -f : f;
}

// Tile anchor for samples i0 + k, k in [0, L): (U0, V, 2 pi D2, 2 pi D3) with
// U0, V the 32-bit rounded P and D1 and the FP32 small-term coefficients, from
//   P  = E0 + i0 (E1 + i0 (E2 + i0 E3)),  D1 = E1 + i0 (2 E2 + 3 i0 E3),
//   D2 = E2 + 3 i0 E3  (exact mod 2^128).
__device__ __forceinline__ uint4 make_anchor(const Poly& P, uint64_t i0) {
  const u128 e3i = mul_u128_u64(P.e[3], i0);
  const u128 Pp = P.e[0] + mul_u128_u64(P.e[1] + mul_u128_u64(P.e[2] + e3i, i0), i0);
  const u128 e3i3 = e3i + (e3i << 1);
  const u128 D1 = P.e[1] + mul_u128_u64((P.e[2] << 1) + e3i3, i0);
  const u128 D2 = P.e[2] + e3i3;
  const u128 half = ((u128)1) << 95;
  const uint32_t U0 = (uint32_t)((Pp + half) >> 96);
  const uint32_t V = (uint32_t)((D1 + half) >> 96);
  const float e2 = i64_to_f32((long long)(uint64_t)(D2 >> 64)) * TWO_PI_2M64;
  const float e3 = i64_to_f32((long long)(uint64_t)(P.e[3] >> 64)) * TWO_PI_2M64;
  return make_uint4(U0, V, __float_as_uint(e2), __float_as_uint(e3));
}

// ---------------------------------------------------------------------------
// Full model (7 parameters): the phase polynomial in the sample index gains
// E4 i^4, and the amplitude is linear in the sample index.

// Coefficient E_k (k = 0..4) of full-model candidate th for the block's time
// base (the Taylor coefficients of p at t0, times h^k):
//   E4 = f3 h^4/24,  E3 = (f2 + f3 t0) h^3/6,  E2 = (f1 + f2 t0 + f3 t0^2/2) h^2/2,
//   E1 = (f0 + f1 t0 + f2 t0^2/2 + f3 t0^3/6) h,
//   E0 = phi0/(2 pi) + f0 t0 + f1 t0^2/2 + f2 t0^3/6 + f3 t0^4/24.
__device__ __forceinline__ double poly_coef_full(const double* th, const BlockArgs& b, int k) {
  const double phi0 = th[1], f0 = th[2], f1 = th[3], f2 = th[4], f3 = th[6];
  if (k == 4) return f3 * b.h4_24;
  if (k == 3) return fma(f3, b.t0, f2) * b.h3_6;
  if (k == 2) return fma(f3, b.t0sq_2, fma(f2, b.t0, f1)) * b.h2_2;
  if (k == 1) return fma(f3, b.t0cu_6, fma(f2, b.t0sq_2, fma(f1, b.t0, f0))) * b.h;
  return fma(f3, b.t0qu_24, fma(f2, b.t0cu_6, fma(f1, b.t0sq_2, fma(f0, b.t0, phi0 * INV_TWO_PI))));
}

// The full model's amplitude A + A1 t at sample i as A0 + i a1h (FP32):
// A0 = A + A1 t0, a1h = A1 h.
struct AmpTerms {
  float A0, a1h;
};
__device__ __forceinline__ AmpTerms full_amp(const double* th, double t0, double h) {
  return {__double2float_rn(fma(th[5], t0, th[0])), __double2float_rn(th[5] * h)};
}

// Inside a lane's run of M samples kc + m' (|m'| <= M/2) the full model's
// small phase terms are the Taylor expansion S0 + S1 m' + S2 m'^2 + S3 m'^3 +
// S4 m'^4 about kc. Dropping S3 m'^3 + S4 m'^4 errs by at most
// 2 pi ((M/2)^3 |S3| + (M/2)^4 |S4|) rad, with |S4| = |E4| and, the anchors
// sitting at tile centres (i0 + L/2 <= n + L) and |kc| <= L/2,
// |S3| <= |E3| + 4 |E4| (n + 2 L); a candidate keeps them when that bound
// exceeds 2^-24 rad (NaN keeps them too). With the block's constants
// quartic_k3 = 2 pi (M/2)^3 and quartic_k4 = 2 pi ((M/2)^4 + 4 (n + 2 L) (M/2)^3)
// the bound is quartic_k3 |E3| + quartic_k4 |E4|: one multiply and one FMA.
__device__ __forceinline__ bool quartic_needed(double E3, double E4, const BlockArgs& b) {
  const double bound = fma(b.quartic_k4, fabs(E4), b.quartic_k3 * fabs(E3));
  return !(bound <= 5.9604644775390625e-08);
}

// Full-model tile anchor for samples i0 + k, i0 the tile's centre sample
// (k in [-L/2, L/2)): exact mod 2^128,
//   p(i0 + k) = P + D1 k + D2 k^2 + D3 k^3 + E4 k^4,
//   P  = E0 + i0 (E1 + i0 (E2 + i0 (E3 + i0 E4))),
//   D1 = E1 + i0 (2 E2 + i0 (3 E3 + 4 i0 E4)),
//   D2 = E2 + i0 (3 E3 + 6 i0 E4),  D3 = E3 + 4 i0 E4;
// first word (U0, V, 2 pi D2, 2 pi D3) as in make_anchor, second
// (2 pi E4, -amplitude at i0, -a1h, 0).
__device__ __forceinline__ void make_anchor_full(const u128 (&e)[5], uint64_t i0, float A0, float a1h, uint4* out) {
  const u128 e4i = mul_u128_u64(e[4], i0);
  const u128 e3x3 = e[3] + (e[3] << 1);
  const u128 Pp = e[0] + mul_u128_u64(e[1] + mul_u128_u64(e[2] + mul_u128_u64(e[3] + e4i, i0), i0), i0);
  const u128 D1 = e[1] + mul_u128_u64((e[2] << 1) + mul_u128_u64(e3x3 + (e4i << 2), i0), i0);
  const u128 D2 = e[2] + mul_u128_u64(e3x3 + (e4i << 2) + (e4i << 1), i0);
  const u128 D3 = e[3] + (e4i << 2);
  const u128 half = ((u128)1) << 95;
  const uint32_t U0 = (uint32_t)((Pp + half) >> 96);
  const uint32_t V = (uint32_t)((D1 + half) >> 96);
  const float d2 = i64_to_f32((long long)(uint64_t)(D2 >> 64)) * TWO_PI_2M64;
  const float d3 = i64_to_f32((long long)(uint64_t)(D3 >> 64)) * TWO_PI_2M64;
  const float d4 = i64_to_f32((long long)(uint64_t)(e[4] >> 64)) * TWO_PI_2M64;
  const float nAt = -fmaf((float)i0, a1h, A0);
  out[0] = make_uint4(U0, V, __float_as_uint(d2), __float_as_uint(d3));
  out[1] = make_uint4(__float_as_uint(d4), __float_as_uint(nAt), __float_as_uint(-a1h), 0u);
}

// Exponent k of the fixed-point SSE accumulator of a candidate: every
// partial and the total are at most B = n (smax + |A|)^2, and k is chosen so
// that B * 2^k < 2^(bits+1). Computed in FP32 with a factor-2 margin for
// rounding (B_f in [2^(e-1), 2^e) gives B < 2^(e+1), k = bits - e).
// The objective uses bits = 60; the DE uses 53 and keeps 8 low bits of each
// 64-bit accumulator for the arrival count.
constexpr int SSE_BITS_OBJ = 60;
constexpr int SSE_BITS_DE = 53;
__device__ __forceinline__ int sse_scale_exp(int64_t n, float smax, float absA, int bits) {
  const float a = smax + absA;
  float B = (float)n * a * a;
  if (!(B > 1e-30f)) B = 1e-30f;
  const int e = (int)((__float_as_uint(B) >> 23) & 0xff) - 126;  // B in [2^(e-1), 2^e)
  int k = bits - e;
  if (k > 120) k = 120;
  if (k < -120) k = -120;
  return k;
}

// acc * 2^-k as a double, exactly as ldexp would (acc < 2^61, |k| <= 120).
__device__ __forceinline__ double fixed_to_double(unsigned long long acc, int k) {
  if (acc == 0ull) return 0.0;
  const double v = (double)(long long)acc;
  return __longlong_as_double(__double_as_longlong(v) - ((long long)k << 52));
}

__device__ __forceinline__ float exp2_int_f(int k) { return __int_as_float((k + 127) << 23); }

// The full model's exponent: |A + A1 t| <= |A0| + |a1h| n over the block.
__device__ __forceinline__ int full_scale_exp(AmpTerms a, int64_t n, float smax, int bits) {
  return sse_scale_exp(n, smax, fabsf(a.A0) + fabsf(a.a1h) * (float)n, bits);
}

// Objectives (Sec. 2.2): the chi-square of Eq. 2-2-4 and the correlation
// objective of Eq. 2-2-5 with the constant-amplitude model of Eq. 2-2-6,
//   cor = sum_i s_i A cos(phi_i),  F_cor = 1 / (atan(cor) + pi/2),
// "cor" read as the unnormalised cross-correlation (the paper's F_cor tends
// to 1/pi at the fit, which a normalised coefficient cannot reach).
constexpr int OBJ_CHI2 = 0;
constexpr int OBJ_COR = 1;

// Fixed-point exponent of a candidate's sum S = sum_i s_i cos(phi_i), signed:
// |S| <= n smax = B, and k is chosen so that B 2^k < 2^(bits+1) (bits is one
// less than for the unsigned chi-square sums, for the sign).
constexpr int COR_BITS_OBJ = 59;
constexpr int COR_BITS_DE = 52;
__device__ __forceinline__ int cor_scale_exp(int64_t n, float smax, int bits) {
  float B = (float)n * smax;
  if (!(B > 1e-30f)) B = 1e-30f;
  const int e = (int)((__float_as_uint(B) >> 23) & 0xff) - 126;  // B in [2^(e-1), 2^e)
  int k = bits - e;
  if (k > 120) k = 120;
  if (k < -120) k = -120;
  return k;
}

// A signed fixed-point sum acc * 2^-k as a double (|acc| < 2^62, |k| <= 120).
__device__ __forceinline__ double signed_fixed_to_double(long long acc, int k) {
  if (acc == 0) return 0.0;
  const double v = (double)acc;
  return __longlong_as_double(__double_as_longlong(v) - ((long long)k << 52));
}

// Eq. 2-2-5 from the candidate's amplitude and its sum S = sum_i s_i cos(phi_i).
__device__ __forceinline__ double cor_objective_value(double A, double S) {
  return 1.0 / (atan(A * S) + 1.5707963267948966192);
}

// ---------------------------------------------------------------------------
// Warp reduce-scatter of N per-lane values (N a power of two <= 32): returns
// the full-warp sum of value index lane / (32 / N); the 32 / N consecutive
// lanes that share an index all hold that sum. log2(N) halving exchanges
// (N - 1 shuffles) followed by an all-reduce over the remaining lane bits.
template <int N, typename T>
__device__ __forceinline__ T warp_reduce_scatter(const T (&v)[N], int lane) {
  T cur[N];
#pragma unroll
  for (int j = 0; j < N; ++j) cur[j] = v[j];
  int off = 16;
#pragma unroll
  for (int n = N; n > 1; n >>= 1) {
    const bool bit = lane & off;
#pragma unroll
    for (int j = 0; j < n / 2; ++j) {
      const T keep = bit ? cur[n / 2 + j] : cur[j];
      const T send = bit ? cur[j] : cur[n / 2 + j];
      cur[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
    off >>= 1;
  }
  T z = cur[0];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1)
    if (o <= off) z += __shfl_xor_sync(0xffffffffu, z, o);
  return z;
}

// ---------------------------------------------------------------------------
// Sample staging: one bulk (TMA) copy global -> shared completed on an
// mbarrier, then conversion to the compute type with the scale applied.

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait for phase 0 of `mbar`; true if it completed.
__device__ __forceinline__ bool mbar_wait_phase0(uint64_t* mbar, uint64_t timeout_ns) {
  const uint64_t t_start = globaltimer_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(mbar))
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t_start > timeout_ns) return false;
  }
}

// All threads call. Copies `bytes` (multiple of 16, both addresses 16-byte
// aligned) from `src` to `dst`. Returns false if the bounded wait expired.
// extra_tx (0 in normal use) is added to the byte count the mbarrier expects
// without any copy to supply it, so the wait cannot complete and runs out:
// the test of this wait's limit. The missing bytes are then signalled by the
// thread itself and the copies that did run are waited for (bounded again),
// so none is still in flight when the CTA returns.
__device__ __forceinline__ bool bulk_stage(void* dst, const void* src, uint32_t bytes, uint64_t* mbar,
                                           uint64_t timeout_ns, uint32_t extra_tx = 0) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"(bytes + extra_tx)
                 : "memory");
    const uint32_t CHUNK = 32768;
    for (uint32_t off = 0; off < bytes; off += CHUNK) {
      const uint32_t sz = (bytes - off) < CHUNK ? (bytes - off) : CHUNK;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32((char*)dst + off)),
          "l"((const char*)src + off), "r"(sz), "r"(smem_u32(mbar))
          : "memory");
    }
    const int ok = mbar_wait_phase0(mbar, timeout_ns) ? 1 : 0;
    bool complete = ok != 0;
    if (!ok && extra_tx) {
      // the injected shortfall: account for it, then wait for the real copies
      asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(extra_tx)
                   : "memory");
      complete = mbar_wait_phase0(mbar, timeout_ns);
    }
    // once the phase completed, invalidate so the next staging can re-initialise it
    if (complete) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(mbar)) : "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Physical value of stored sample i of a raw buffer.
__device__ __forceinline__ double load_physical(const void* raw, int dtype, int64_t i, double scale) {
  switch (dtype) {
    case 0: return (double)((const int8_t*)raw)[i] * scale;
    case 1: return (double)((const int16_t*)raw)[i] * scale;
    case 2: return (double)__half2float(((const __half*)raw)[i]) * scale;
    case 3: return (double)((const float*)raw)[i] * scale;
    default: return ((const double*)raw)[i] * scale;
  }
}

}  // namespace pt
