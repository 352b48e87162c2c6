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
constexpr int M = 8;             // samples per lane per tile
constexpr int L = 32 * M;        // samples per tile
constexpr int CG = 8;            // candidates per work item
constexpr int NP_MAX = 128;      // largest population / candidate batch per CTA

constexpr double TWO_PI = 2.0 * 3.14159265358979323846;
constexpr double INV_TWO_PI = 0.15915494309189533577;
// 2 pi / 2^32 and 2 pi / 2^64 as FP32 scale factors of fixed-point phases
constexpr float TWO_PI_2M32 = 1.46291807926715968e-09f;
constexpr float TWO_PI_2M64 = 3.40612158008655460e-19f;

// Status written by a kernel into its error word (0 = OK).
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = 1;   // a bounded wait expired

// Per-block constants shared by all kernels.
struct BlockArgs {
  const void* samples;   // device; zero-padded to a multiple of L samples
  int64_t n;             // valid samples
  int64_t ntiles;        // ceil(n / L)
  int dtype;             // PT_I8 .. PT_F64
  int esize;             // bytes per stored sample
  double scale;          // physical = scale * stored
  double smax;           // max |physical sample|
  double t0, h;          // t_i = t0 + i h
  double t0sq_2, t0cu_6; // t0^2/2, t0^3/6
  double h2_2, h3_6;     // h^2/2, h^3/6
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
struct DeControls {
  double lo[D], hi[D];
  double F;
  uint32_t cr_thr;   // crossover if word < cr_thr
  int cr_all;        // CR >= 1
  int periodic;      // phi0 range spans the full circle
  uint2 key;         // Philox key (seed lo, seed hi)
  uint32_t block_id;
};

// Generation-0 individual: uniform inside the bounds.
__device__ __forceinline__ void de_init(const DeControls& dc, int i, double* xi) {
  uint32_t w[12];
  de_draw12(dc.key, dc.block_id, 0u, (uint32_t)i, w);
#pragma unroll
  for (int j = 0; j < D; ++j)
    xi[j] = __dadd_rn(dc.lo[j], __dmul_rn(u53(w[2 * j], w[2 * j + 1]), __dsub_rn(dc.hi[j], dc.lo[j])));
}

// DE/rand/1/bin trial of individual i at generation gen >= 1 from population x (np x 5).
// FP64 operations are written out with _rn intrinsics so no contraction
// changes a rounding: the trial is bit-identical to a plain IEEE evaluation.
__device__ __forceinline__ void de_trial(const DeControls& dc, const double* x, int np, int i, uint32_t gen,
                                         double* ui) {
  uint32_t w[12];
  de_draw12(dc.key, dc.block_id, gen, (uint32_t)i, w);
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
  const uint32_t jrand = lemire(w[3], (uint32_t)D);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double parent = x[i * D + j];
    const bool take = (uint32_t)j == jrand || dc.cr_all || w[4 + j] < dc.cr_thr;
    double u = parent;
    if (take) {
      double v = __dadd_rn(x[r[0] * D + j], __dmul_rn(dc.F, __dsub_rn(x[r[1] * D + j], x[r[2] * D + j])));
      if (j == 1 && dc.periodic) {
        const double k = floor(__ddiv_rn(__dsub_rn(v, dc.lo[j]), TWO_PI));
        v = __dsub_rn(v, __dmul_rn(k, TWO_PI));
      } else if (v < dc.lo[j]) {
        v = __dmul_rn(__dadd_rn(dc.lo[j], parent), 0.5);
      } else if (v > dc.hi[j]) {
        v = __dmul_rn(__dadd_rn(dc.hi[j], parent), 0.5);
      }
      u = v;
    }
    ui[j] = u;
  }
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

// E0..E3 of candidate th = (A, phi0, f0, f1, f2) for the block's time base.
__device__ __forceinline__ Poly make_poly(const double* th, const BlockArgs& b) {
  const double phi0 = th[1], f0 = th[2], f1 = th[3], f2 = th[4];
  Poly P;
  const double E3 = f2 * b.h3_6;
  const double E2 = fma(f2, b.t0, f1) * b.h2_2;
  const double E1 = fma(f2, b.t0sq_2, fma(f1, b.t0, f0)) * b.h;
  // E0 = phi0/(2 pi) + f0 t0 + f1 t0^2/2 + f2 t0^3/6
  const double E0 = fma(f2, b.t0cu_6, fma(f1, b.t0sq_2, fma(f0, b.t0, phi0 * INV_TWO_PI)));
  P.e[0] = frac128(E0);
  P.e[1] = frac128(E1);
  P.e[2] = frac128(E2);
  P.e[3] = frac128(E3);
  return P;
}

// Tile anchor for samples i0 + k, k in [0, L): (U0, V, 2 pi D2, 2 pi D3) with
// U0, V the 32-bit rounded P and D1 and the FP32 small-term coefficients.
__device__ __forceinline__ uint4 make_anchor(const Poly& P, uint64_t i0) {
  const u128 I = i0, I2 = I * I, I3 = I2 * I;
  const u128 Pp = P.e[0] + P.e[1] * I + P.e[2] * I2 + P.e[3] * I3;
  const u128 D1 = P.e[1] + ((P.e[2] * I) << 1) + (u128)3 * P.e[3] * I2;
  const u128 D2 = P.e[2] + (u128)3 * P.e[3] * I;
  const u128 half = ((u128)1) << 95;
  const uint32_t U0 = (uint32_t)((Pp + half) >> 96);
  const uint32_t V = (uint32_t)((D1 + half) >> 96);
  const float e2 = (float)(long long)(uint64_t)(D2 >> 64) * TWO_PI_2M64;
  const float e3 = (float)(long long)(uint64_t)(P.e[3] >> 64) * TWO_PI_2M64;
  return make_uint4(U0, V, __float_as_uint(e2), __float_as_uint(e3));
}

// Exponent k of the fixed-point SSE accumulator of a candidate: every
// partial and the total are below n (smax + |A|)^2 < 2^(61-k) * 2^k ... i.e.
// scaled values stay below 2^61.
__device__ __forceinline__ int sse_scale_exp(int64_t n, double smax, double A) {
  const double a = smax + fabs(A);
  double B = (double)n * a * a;
  if (!(B > 1e-200)) B = 1e-200;
  int e;
  frexp(B, &e);  // B < 2^e
  int k = 61 - e;
  if (k > 120) k = 120;
  if (k < -120) k = -120;
  return k;
}

__device__ __forceinline__ float exp2_int_f(int k) { return __int_as_float((k + 127) << 23); }

// ---------------------------------------------------------------------------
// Warp reduce-scatter of 8 per-lane values: returns the full-warp sum of value
// index (lane >> 2) & 7 (lanes 4c..4c+3 hold the sum of value c).
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter8(const T (&v)[8], int lane) {
  const unsigned FULL = 0xffffffffu;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  T w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T keep = b4 ? v[4 + j] : v[j];
    const T send = b4 ? v[j] : v[4 + j];
    w[j] = keep + __shfl_xor_sync(FULL, send, 16);
  }
  T y[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T keep = b3 ? w[2 + j] : w[j];
    const T send = b3 ? w[j] : w[2 + j];
    y[j] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  T z = (b2 ? y[1] : y[0]) + __shfl_xor_sync(FULL, b2 ? y[0] : y[1], 4);
  z += __shfl_xor_sync(FULL, z, 2);
  z += __shfl_xor_sync(FULL, z, 1);
  return z;
}

// ---------------------------------------------------------------------------
// Sample staging: one bulk (TMA) copy global -> shared completed on an
// mbarrier, then conversion to the compute type with the scale applied.

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// All threads call. Copies `bytes` (multiple of 16, both addresses 16-byte
// aligned) from `src` to `dst`. Returns false if the bounded wait expired.
__device__ __forceinline__ bool bulk_stage(void* dst, const void* src, uint32_t bytes, uint64_t* mbar,
                                           uint64_t timeout_ns) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
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
    // bounded wait for phase 0
    const uint64_t t_start = globaltimer_ns();
    int ok = 0;
    while (true) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(smem_u32(mbar))
          : "memory");
      if (done) {
        ok = 1;
        break;
      }
      if (globaltimer_ns() - t_start > timeout_ns) break;
    }
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
