// Kernels of the phase-tracking hot path (arxiv 1906.10598, Sec. 1.2-2.2):
//   k_absmax      max |stored sample| of a loaded block (sets the SSE fixed-point scale)
//   k_objective   Eq. 2-2-4 for a fixed candidate set (tiles x candidate batches)
//   k_finalize    fixed-point accumulators -> FP64 SSE
//   k_de          persistent DE solve of a group's blocks (Table 3-1-1 controls and strategies)
//
// Work decomposition shared by the objective and DE kernels: a CTA owns a
// contiguous range of 256-sample tiles, staged once into shared memory by a
// bulk (TMA) copy and converted to the compute type; a work item is one tile
// x CG candidates (CG = 4, 8 or 16), run by one warp with 8 consecutive samples per lane in
// registers. Per-item FP32 sums are reduced across the warp and added, as
// 64-bit fixed point with a per-candidate scale, to shared and then global
// accumulators. Integer addition is exact and associative, so the SSE does not
// depend on the launch shape, the CTA count or the order of completion.
#pragma once

#include <climits>

#include "pt_device.cuh"

namespace pt {

constexpr int NT = 512;        // threads per CTA of the DE kernels
constexpr int NT_OBJ = 256;    // threads per CTA of the objective kernel, OBJ_CTAS of them per SM
constexpr int OBJ_CTAS = 2;
constexpr int CAND_BYTES = 64; // per-candidate prepared data in shared memory
// The full model's per-candidate data: E0..E4 (5 x 16 B), then A0 and a1h (FP32).
constexpr int CAND_BYTES_FULL = 96;
__host__ __device__ constexpr int cand_bytes(int model) { return model == MODEL_FULL ? CAND_BYTES_FULL : CAND_BYTES; }
// 16-byte anchor words per candidate and tile
__host__ __device__ constexpr int anchor_words(int model) { return model == MODEL_FULL ? 2 : 1; }

enum Tier { TIER_F64 = 0, TIER_PLAIN = 1, TIER_DF32 = 2, TIER_F32 = 3 };

__host__ __device__ constexpr bool tier_uses_f64_samples(int tier) { return tier == TIER_PLAIN; }

// ---------------------------------------------------------------------------
// double-float (pairs of FP32) arithmetic for the DF32 tier
struct dfloat {
  float hi, lo;
};
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat df_from_double(double v) {
  const float hi = __double2float_rn(v);
  return {hi, __double2float_rn(v - (double)hi)};
}

// ---------------------------------------------------------------------------
// Per-candidate preparation (one thread per candidate).
//   TIER_F64:   Poly (4 x u128) for the tile anchors
//   TIER_PLAIN: double[5] = A, phi0/(2 pi), f0, f1/2, f2/6
//   TIER_DF32:  dfloat[4] = c0..c3 (cycles, seconds), A in negA
//   TIER_F32:   float[4]  = c0..c3
// MODEL_FULL (comparison tiers): the phase coefficients gain f3/24 and the
// amplitude terms follow them; the exponent is the full model's.
//   TIER_PLAIN: double[7] = A, A1, phi0/(2 pi), f0, f1/2, f2/6, f3/24
//   TIER_DF32:  dfloat[5] = phi0/(2 pi), f0, f1/2, f2/6, f3/24, then float A, A1
//   TIER_F32:   float[5] = the same, then float A, A1
template <int TIER, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__device__ __forceinline__ void prep_candidate(const double* th, const BlockArgs& b, unsigned char* cdata,
                                               float* negA, int* kexp, int kbits) {
  if constexpr (MODEL == MODEL_FULL) {
    *negA = 0.f;
    *kexp = full_scale_exp(full_amp(th, b.t0, b.h), b.n, b.smax_f, kbits);
    const double pc[5] = {th[1] * INV_TWO_PI, th[2], th[3] * 0.5, th[4] * (1.0 / 6.0), th[6] * (1.0 / 24.0)};
    if (TIER == TIER_PLAIN) {
      double* c = reinterpret_cast<double*>(cdata);
      c[0] = th[0];
      c[1] = th[5];
      for (int k = 0; k < 5; ++k) c[2 + k] = pc[k];
    } else if (TIER == TIER_DF32) {
      dfloat* c = reinterpret_cast<dfloat*>(cdata);
      for (int k = 0; k < 5; ++k) c[k] = df_from_double(pc[k]);
      reinterpret_cast<float*>(cdata + 40)[0] = __double2float_rn(th[0]);
      reinterpret_cast<float*>(cdata + 40)[1] = __double2float_rn(th[5]);
    } else {
      float* c = reinterpret_cast<float*>(cdata);
      for (int k = 0; k < 5; ++k) c[k] = __double2float_rn(pc[k]);
      c[5] = __double2float_rn(th[0]);
      c[6] = __double2float_rn(th[5]);
    }
    return;
  }
  const float Af = __double2float_rn(th[0]);
  *negA = -Af;
  *kexp = OBJ == OBJ_COR ? cor_scale_exp(b.n, b.smax_f, kbits) : sse_scale_exp(b.n, b.smax_f, fabsf(Af), kbits);
  if (TIER == TIER_F64) {
    u128* e = reinterpret_cast<u128*>(cdata);
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = poly_term(th, b, k);
  } else if (TIER == TIER_PLAIN) {
    double* c = reinterpret_cast<double*>(cdata);
    c[0] = th[0];
    c[1] = th[1] * INV_TWO_PI;
    c[2] = th[2];
    c[3] = th[3] * 0.5;
    c[4] = th[4] * (1.0 / 6.0);
  } else if (TIER == TIER_DF32) {
    dfloat* c = reinterpret_cast<dfloat*>(cdata);
    c[0] = df_from_double(th[1] * INV_TWO_PI);
    c[1] = df_from_double(th[2]);
    c[2] = df_from_double(th[3] * 0.5);
    c[3] = df_from_double(th[4] * (1.0 / 6.0));
  } else {
    float* c = reinterpret_cast<float*>(cdata);
    c[0] = __double2float_rn(th[1] * INV_TWO_PI);
    c[1] = __double2float_rn(th[2]);
    c[2] = __double2float_rn(th[3] * 0.5);
    c[3] = __double2float_rn(th[4] * (1.0 / 6.0));
  }
}

template <int MODEL = MODEL_CUBIC>
__device__ __forceinline__ void prep_zero(unsigned char* cdata, float* negA, int* kexp) {
  *negA = 0.f;
  *kexp = 0;
  uint4* p = reinterpret_cast<uint4*>(cdata);
#pragma unroll
  for (int k = 0; k < cand_bytes(MODEL) / 16; ++k) p[k] = make_uint4(0, 0, 0, 0);
}

// Prepare candidates [0, nc) of `cands` (rows of model_dim(MODEL) doubles) padded to npad.
// The default tier spreads the four FP64 polynomial terms and the amplitude
// over separate threads so the 1/64-rate FP64 work is spread across all
// warps of the CTA, and flags in cub[c] the candidates whose cubic term must
// stay exact (cubic_needed). The full model (default tier, chi-square)
// spreads its five terms and the amplitude/flag/exponent work the same way.
// Tasks are taken from `first` in steps of `stride` (a thread range of the
// CTA); with a list, only the candidates list[0 .. nlist) (all below nc) are
// prepared, with one >= 0 only candidate `one`. No barrier.
template <int TIER, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__device__ void prep_range(const double* cands, int nc, int npad, const BlockArgs& b, unsigned char* cdata,
                           float* negA, int* kexp, unsigned char* cub, int kbits, int first, int stride,
                           const unsigned char* list = nullptr, int nlist = 0, int one = -1) {
  const int m = one >= 0 ? 1 : list ? nlist : npad;
  if constexpr (MODEL == MODEL_FULL && TIER == TIER_F64) {
    for (int t = first; t < 6 * m; t += stride) {
      const int k = t / m, i = t - k * m;
      const int c = one >= 0 ? one : list ? (int)list[i] : i;
      const double* th = cands + c * DF;
      unsigned char* cd = cdata + c * CAND_BYTES_FULL;
      if (k < 4) {
        reinterpret_cast<u128*>(cd)[k] = frac128(c < nc ? poly_coef_full(th, b, k) : 0.0);
      } else if (k == 4) {
        // E4, and the quartic flag from E4 and a second copy of E3 (two FP64
        // operations) on the same thread
        const double E4 = c < nc ? poly_coef_full(th, b, 4) : 0.0;
        reinterpret_cast<u128*>(cd)[4] = frac128(E4);
        cub[c] = c < nc && quartic_needed(poly_coef_full(th, b, 3), E4, b) ? 1 : 0;
      } else if (c < nc) {
        const AmpTerms am = full_amp(th, b.t0, b.h);
        reinterpret_cast<float*>(cd + 80)[0] = am.A0;
        reinterpret_cast<float*>(cd + 80)[1] = am.a1h;
        negA[c] = 0.f;
        kexp[c] = full_scale_exp(am, b.n, b.smax_f, kbits);
      } else {
        reinterpret_cast<float*>(cd + 80)[0] = 0.f;
        reinterpret_cast<float*>(cd + 80)[1] = 0.f;
        negA[c] = 0.f;
        kexp[c] = 0;
      }
    }
  } else if constexpr (TIER == TIER_F64) {
    for (int t = first; t < 5 * m; t += stride) {
      const int k = t / m, i = t - k * m;
      const int c = one >= 0 ? one : list ? (int)list[i] : i;
      if (k < 4) {
        const double E = c < nc ? poly_coef(cands + c * D, b, k) : 0.0;
        reinterpret_cast<u128*>(cdata + c * CAND_BYTES)[k] = frac128(E);
        if (k == 3) cub[c] = cubic_needed(E) ? 1 : 0;
      } else if (c < nc) {
        const float Af = __double2float_rn(cands[c * D]);
        negA[c] = -Af;
        kexp[c] = OBJ == OBJ_COR ? cor_scale_exp(b.n, b.smax_f, kbits) : sse_scale_exp(b.n, b.smax_f, fabsf(Af), kbits);
      } else {
        negA[c] = 0.f;
        kexp[c] = 0;
      }
    }
  } else {
    constexpr int CB = cand_bytes(MODEL);
    for (int i = first; i < m; i += stride) {
      const int c = one >= 0 ? one : list ? (int)list[i] : i;
      if (c < nc)
        prep_candidate<TIER, OBJ, MODEL>(cands + c * model_dim(MODEL), b, cdata + c * CB, negA + c, kexp + c, kbits);
      else prep_zero<MODEL>(cdata + c * CB, negA + c, kexp + c);
      cub[c] = 0;
    }
  }
}

// All of the CTA prepares candidates [0, nc) padded to npad; ends with __syncthreads().
template <int TIER, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__device__ void prep_all(const double* cands, int nc, int npad, const BlockArgs& b, unsigned char* cdata,
                         float* negA, int* kexp, unsigned char* cub, int kbits) {
  prep_range<TIER, OBJ, MODEL>(cands, nc, npad, b, cdata, negA, kexp, cub, kbits, threadIdx.x, blockDim.x);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Work items: one warp, one 256-sample tile, CGV candidates, 8 samples per lane.

// Default tier, one candidate, exact cubic: the lane's phase is anchored at
// its centre sample kc in fixed point, and its M samples kc + m' follow in
// FP32 from the exact expansion of the small terms about kc,
//   E2 k^2 + E3 k^3 = S0 + m' S1 + m'^2 S2 + m'^3 E3,
//   S0 = E2 kc^2 + E3 kc^3,  S1 = 2 E2 kc + 3 E3 kc^2,  S2 = E2 + 3 E3 kc,
// so x = xc + m' Vc + m'^2 S2 + m'^3 E3 with xc = 2 pi frac(U0 + kc V) + S0
// and Vc = 2 pi V + S1: three FFMAs per sample (none at the centre). MASKED
// zeroes the residuals of samples at or past nvalid (the ragged last tile).
// OBJ_COR accumulates s_i cos(phi_i) instead of the squared residual.
template <bool MASKED, int OBJ>
__device__ __forceinline__ float cand_exact(const float (&s)[M], uint4 a, float nA, int lane, int nvalid) {
  const int kci = lane * M + M / 2;
  const float kc = (float)kci, kc2 = kc * kc;
  const uint32_t V = a.y;
  const float E2 = __uint_as_float(a.z), E3 = __uint_as_float(a.w);
  const float S0 = fmaf(E3, kc2 * kc, E2 * kc2);
  const float S1 = fmaf(E3, 3.0f * kc2, E2 * (2.0f * kc));
  const float S2 = fmaf(E3, 3.0f * kc, E2);
  const float xc = fmaf((float)(int)(a.x + (uint32_t)kci * V), TWO_PI_2M32, S0);
  const float Vc = fmaf((float)(int)V, TWO_PI_2M32, S1);
  float sum = 0.f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float mp = (float)(m - M / 2);
    const float x = (m == M / 2) ? xc : fmaf(mp, Vc, fmaf(mp * mp, S2, fmaf(mp * mp * mp, E3, xc)));
    const float cv = __cosf(x);
    if (OBJ == OBJ_COR) {
      // samples past nvalid are the zero padding of the staged tile
      sum = fmaf(s[m], cv, sum);
    } else {
      float r = fmaf(nA, cv, s[m]);
      if (MASKED) r = (lane * M + m < nvalid) ? r : 0.f;
      sum = fmaf(r, r, sum);
    }
  }
  return sum;
}

// Default tier, one candidate, cubic folded (the candidate is not flagged by
// cubic_needed): the lane's phase is anchored once at its centre sample kc in
// fixed point, and its M samples kc + m' follow in FP32 as
//   x = xc + m' Vc + m'^2 E2c,  xc = 2 pi frac(U0 + kc V) + E2c kc^2,
//   Vc = 2 pi V + 2 kc E2c,     E2c = E2 + kc E3,
// two FFMAs with constant m' per sample instead of the fixed-point walk
// (none at the centre itself). |x| stays below (1 + M) pi.
template <int OBJ>
__device__ __forceinline__ float cand_fold(const float (&s)[M], uint4 a, float nA, int lane) {
  const int kci = lane * M + M / 2;
  const float kc = (float)kci;
  const uint32_t V = a.y;
  const float E2 = __uint_as_float(a.z), E3 = __uint_as_float(a.w);
  const float E2c = fmaf(E3, kc, E2);
  const float xc = fmaf((float)(int)(a.x + (uint32_t)kci * V), TWO_PI_2M32, E2c * (kc * kc));
  const float Vc = fmaf((float)(int)V, TWO_PI_2M32, E2c * (2.0f * kc));
  float sum = 0.f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float mp = (float)(m - M / 2);
    const float x = (m == M / 2) ? xc : fmaf(mp, Vc, fmaf(mp * mp, E2c, xc));
    const float cv = __cosf(x);
    if (OBJ == OBJ_COR) {
      sum = fmaf(s[m], cv, sum);
    } else {
      const float r = fmaf(nA, cv, s[m]);
      sum = fmaf(r, r, sum);
    }
  }
  return sum;
}

// Default-tier items. A candidate's partial over a tile depends only on the
// candidate and the tile: full tiles use cand_fold unless the candidate is
// flagged (flags: its CGV bytes, nonzero = keep the exact cubic), the ragged
// last tile always uses cand_exact.
template <int CGV, bool MASKED, int OBJ>
__device__ __forceinline__ void item_f64(const float (&s)[M], const uint4* anc_i, const float* negA_g, int lane,
                                         int nvalid, float (&acc)[CGV]) {
#pragma unroll
  for (int c = 0; c < CGV; ++c) acc[c] = cand_exact<MASKED, OBJ>(s, anc_i[c], negA_g[c], lane, nvalid);
}
// The CGV values -A of an item's candidates (negA_g 16-byte aligned, CGV a
// multiple of 4), in 16-byte loads.
template <int CGV>
__device__ __forceinline__ void load_negA(const float* negA_g, float (&nA)[CGV]) {
#pragma unroll
  for (int c = 0; c < CGV; c += 4) {
    const float4 v = *reinterpret_cast<const float4*>(negA_g + c);
    nA[c] = v.x;
    nA[c + 1] = v.y;
    nA[c + 2] = v.z;
    nA[c + 3] = v.w;
  }
}
template <int CGV, int OBJ>
__device__ __forceinline__ void item_f64_fold(const float (&s)[M], const uint4* anc_i, const float* negA_g, int lane,
                                              float (&acc)[CGV]) {
  float nA[CGV];
  if (OBJ == OBJ_CHI2) load_negA<CGV>(negA_g, nA);
#pragma unroll
  for (int c = 0; c < CGV; ++c) acc[c] = cand_fold<OBJ>(s, anc_i[c], OBJ == OBJ_CHI2 ? nA[c] : 0.f, lane);
}
template <int CGV, int OBJ>
__device__ __forceinline__ void item_f64_mixed(const float (&s)[M], const uint4* anc_i, const float* negA_g,
                                               const unsigned char* flags, int lane, float (&acc)[CGV]) {
#pragma unroll
  for (int c = 0; c < CGV; ++c) {
    if (flags[c]) acc[c] = cand_exact<false, OBJ>(s, anc_i[c], negA_g[c], lane, L);
    else acc[c] = cand_fold<OBJ>(s, anc_i[c], negA_g[c], lane);
  }
}

// Full model, one candidate: anchor words a = (U0, V, 2 pi D2, 2 pi D3) and
// q = (2 pi E4, -amplitude at the tile's centre, -a1h), anchored at the tile's
// centre sample (so kc = lane M + M/2 - L/2 lies in [-L/2, L/2) and the small
// terms stay a quarter of their size at the tile start). The lane's phase is
// anchored at its centre sample kc in fixed point; the small terms
// Q(k) = d2 k^2 + d3 k^3 + d4 k^4 follow from their Taylor expansion about kc,
//   S0 = Q(kc), S1 = Q'(kc), S2 = Q''(kc)/2, S3 = d3 + 4 d4 kc, S4 = d4,
// x = xc + m' Vc + m'^2 S2 [+ m'^3 S3 + m'^4 S4] with xc = 2 pi frac(U0 + kc V)
// + S0 and Vc = 2 pi V + S1; QUARTIC keeps the bracket (quartic_needed). The
// amplitude walks as A_c + m' a1h from the lane centre.
template <bool QUARTIC, bool MASKED>
__device__ __forceinline__ float cand_full(const float (&s)[M], uint4 a, uint4 q, int lane, int nvalid) {
  const int kci = lane * M + M / 2 - L / 2;
  // the lane's weights (the same for every candidate, so computed once per item)
  const float kc = (float)kci, kc2 = kc * kc, kc3 = kc2 * kc, kc4 = kc2 * kc2;
  const uint32_t V = a.y;
  const float d2 = __uint_as_float(a.z), d3 = __uint_as_float(a.w), d4 = __uint_as_float(q.x);
  const float S0 = fmaf(kc4, d4, fmaf(kc3, d3, kc2 * d2));
  const float S1 = fmaf(4.0f * kc3, d4, fmaf(3.0f * kc2, d3, (2.0f * kc) * d2));
  const float S2 = fmaf(6.0f * kc2, d4, fmaf(3.0f * kc, d3, d2));
  const float S3 = fmaf(4.0f * kc, d4, d3);
  const float xc = fmaf((float)(int)(a.x + (uint32_t)kci * V), TWO_PI_2M32, S0);
  const float Vc = fmaf((float)(int)V, TWO_PI_2M32, S1);
  // the anchor holds -A(tile centre) and -a1h
  const float na1 = __uint_as_float(q.z);
  const float nAc = fmaf(kc, na1, __uint_as_float(q.y));
  float sum = 0.f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float mp = (float)(m - M / 2);
    float x = xc;
    if (m != M / 2) {
      x = QUARTIC ? fmaf(mp, Vc, fmaf(mp * mp, S2, fmaf(mp * mp * mp, S3, fmaf(mp * mp * mp * mp, d4, xc))))
                  : fmaf(mp, Vc, fmaf(mp * mp, S2, xc));
    }
    const float cv = __cosf(x);
    const float nA = (m == M / 2) ? nAc : fmaf(mp, na1, nAc);
    float r = fmaf(nA, cv, s[m]);
    if (MASKED) r = (lane * M + m < nvalid) ? r : 0.f;
    sum = fmaf(r, r, sum);
  }
  return sum;
}

// Full-model items: every candidate exact and masked on the ragged last tile;
// on full tiles the flagged candidates keep the quartic terms.
template <int CGV>
__device__ __forceinline__ void item_full_masked(const float (&s)[M], const uint4* anc_i, int lane, int nvalid,
                                                 float (&acc)[CGV]) {
#pragma unroll
  for (int c = 0; c < CGV; ++c) acc[c] = cand_full<true, true>(s, anc_i[2 * c], anc_i[2 * c + 1], lane, nvalid);
}
template <int CGV>
__device__ __forceinline__ void item_full_fold(const float (&s)[M], const uint4* anc_i, int lane, float (&acc)[CGV]) {
#pragma unroll
  for (int c = 0; c < CGV; ++c) acc[c] = cand_full<false, false>(s, anc_i[2 * c], anc_i[2 * c + 1], lane, L);
}
template <int CGV>
__device__ __forceinline__ void item_full_mixed(const float (&s)[M], const uint4* anc_i, const unsigned char* flags,
                                                int lane, float (&acc)[CGV]) {
#pragma unroll
  for (int c = 0; c < CGV; ++c) {
    if (flags[c]) acc[c] = cand_full<true, false>(s, anc_i[2 * c], anc_i[2 * c + 1], lane, L);
    else acc[c] = cand_full<false, false>(s, anc_i[2 * c], anc_i[2 * c + 1], lane, L);
  }
}

// All-FP64 tier: Horner phase in seconds, reduction mod 1, FP64 cospi.
// OBJ_COR accumulates s_i cos(phi_i) (the padding samples are zero).
// MODEL_FULL: the quartic phase and the amplitude A + A1 t.
template <int CGV, bool MASKED, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__device__ __forceinline__ void item_plain(const double (&s)[M], const unsigned char* cdata_g, int lane, int nvalid,
                                           int64_t tstart, const BlockArgs& b, double (&acc)[CGV]) {
#pragma unroll 1
  for (int c = 0; c < CGV; ++c) {
    const double* k = reinterpret_cast<const double*>(cdata_g + c * cand_bytes(MODEL));
    double A, A1 = 0.0, c0, c1, c2, c3, c4 = 0.0;
    if constexpr (MODEL == MODEL_FULL) {
      A = k[0], A1 = k[1], c0 = k[2], c1 = k[3], c2 = k[4], c3 = k[5], c4 = k[6];
    } else {
      A = k[0], c0 = k[1], c1 = k[2], c2 = k[3], c3 = k[4];
    }
    double sum = 0.0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int64_t i = tstart + lane * M + m;
      const double t = fma((double)i, b.h, b.t0);
      const double p = MODEL == MODEL_FULL ? fma(fma(fma(fma(c4, t, c3), t, c2), t, c1), t, c0)
                                           : fma(fma(fma(c3, t, c2), t, c1), t, c0);
      const double r = p - rint(p);
      const double cv = cospi(2.0 * r);
      if (OBJ == OBJ_COR) {
        sum = fma(s[m], cv, sum);
      } else {
        const double Am = MODEL == MODEL_FULL ? fma(A1, t, A) : A;
        double res = fma(-Am, cv, s[m]);
        if (MASKED) res = (lane * M + m < nvalid) ? res : 0.0;
        sum = fma(res, res, sum);
      }
    }
    acc[c] = sum;
  }
}

// Double-float tier: per-sample phase in double-float, FP32 cosine.
template <int CGV, bool MASKED, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__device__ __forceinline__ void item_df32(const float (&s)[M], const unsigned char* cdata_g, const float* negA_g,
                                          int lane, int nvalid, int64_t tstart, dfloat t0d, dfloat hd,
                                          float (&acc)[CGV]) {
#pragma unroll 1
  for (int c = 0; c < CGV; ++c) {
    const dfloat* k = reinterpret_cast<const dfloat*>(cdata_g + c * cand_bytes(MODEL));
    const dfloat c0 = k[0], c1 = k[1], c2 = k[2], c3 = k[3];
    const dfloat c4 = MODEL == MODEL_FULL ? k[4] : dfloat{0.f, 0.f};
    float nA = negA_g[c], A = 0.f, A1 = 0.f;
    if constexpr (MODEL == MODEL_FULL) {
      A = reinterpret_cast<const float*>(cdata_g + c * cand_bytes(MODEL) + 40)[0];
      A1 = reinterpret_cast<const float*>(cdata_g + c * cand_bytes(MODEL) + 40)[1];
    }
    float sum = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int64_t i = tstart + lane * M + m;
      // t = t0 + i h in double-float (i < 2^24 is exact in FP32)
      const dfloat t = df_add(t0d, df_mul({(float)i, 0.f}, hd));
      dfloat p = MODEL == MODEL_FULL ? df_add(df_mul(df_add(df_mul(c4, t), c3), t), c2) : df_add(df_mul(c3, t), c2);
      p = df_add(df_mul(p, t), c1);
      p = df_add(df_mul(p, t), c0);
      const float rh = p.hi - rintf(p.hi);
      const float r = rh + p.lo;
      const float cv = __cosf(r * 6.28318530717958648f);
      if (MODEL == MODEL_FULL) nA = -fmaf(A1, t.hi, A);
      if (OBJ == OBJ_COR) {
        sum = fmaf(s[m], cv, sum);
      } else {
        float res = fmaf(nA, cv, s[m]);
        if (MASKED) res = (lane * M + m < nvalid) ? res : 0.f;
        sum = fmaf(res, res, sum);
      }
    }
    acc[c] = sum;
  }
}

// Naive FP32 tier: Horner phase in seconds in FP32.
template <int CGV, bool MASKED, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__device__ __forceinline__ void item_f32(const float (&s)[M], const unsigned char* cdata_g, const float* negA_g,
                                         int lane, int nvalid, int64_t tstart, float t0f, float hf,
                                         float (&acc)[CGV]) {
#pragma unroll 1
  for (int c = 0; c < CGV; ++c) {
    const float* k = reinterpret_cast<const float*>(cdata_g + c * cand_bytes(MODEL));
    const float c0 = k[0], c1 = k[1], c2 = k[2], c3 = k[3];
    const float c4 = MODEL == MODEL_FULL ? k[4] : 0.f;
    const float A = MODEL == MODEL_FULL ? k[5] : 0.f, A1 = MODEL == MODEL_FULL ? k[6] : 0.f;
    float nA = negA_g[c];
    float sum = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int64_t i = tstart + lane * M + m;
      const float t = fmaf((float)i, hf, t0f);
      const float p = MODEL == MODEL_FULL ? fmaf(fmaf(fmaf(fmaf(c4, t, c3), t, c2), t, c1), t, c0)
                                          : fmaf(fmaf(fmaf(c3, t, c2), t, c1), t, c0);
      const float r = p - rintf(p);
      const float cv = __cosf(r * 6.28318530717958648f);
      if (MODEL == MODEL_FULL) nA = -fmaf(A1, t, A);
      if (OBJ == OBJ_COR) {
        sum = fmaf(s[m], cv, sum);
      } else {
        float res = fmaf(nA, cv, s[m]);
        if (MASKED) res = (lane * M + m < nvalid) ? res : 0.f;
        sum = fmaf(res, res, sum);
      }
    }
    acc[c] = sum;
  }
}

// Candidates per work item of the default tier for a batch of n candidates:
// the width in {16, 8, 4} with the least padded work, each padded candidate
// weighted by the measured cost per candidate of its width on B300 (narrower
// items amortise the per-item anchor loads, reduction and loop over fewer
// candidates: 1.0, 1.1 and 1.4 for 16, 8 and 4).
inline int pick_cg_f64(int n) {
  int best = 16;
  double best_cost = (double)((n + 15) / 16 * 16);
  const int widths[2] = {8, 4};
  const double weight[2] = {1.1, 1.4};
  for (int i = 0; i < 2; ++i) {
    const double cost = (double)((n + widths[i] - 1) / widths[i] * widths[i]) * weight[i];
    if (cost < best_cost) {
      best = widths[i];
      best_cost = cost;
    }
  }
  return best;
}

// Items a warp evaluates per anchor batch (default tier).
constexpr int IPB = 4;

// Whether any of the CGV candidates at `f` (16-byte aligned for CGV = 16)
// carries a cubic_needed flag.
template <int CGV>
__device__ __forceinline__ bool any_flag(const unsigned char* f) {
  if (CGV == 16) {
    const uint4 w = *reinterpret_cast<const uint4*>(f);
    return (w.x | w.y | w.z | w.w) != 0u;
  } else if (CGV == 8) {
    const uint2 w = *reinterpret_cast<const uint2*>(f);
    return (w.x | w.y) != 0u;
  } else {
    return *reinterpret_cast<const uint32_t*>(f) != 0u;
  }
}

// Evaluate candidates [0, ncand) (prepared in cdata/negA/kexp, padded to npad,
// a multiple of CGV) on items [item_lo, item_hi) of the tiles staged from
// tile_begin, whose converted samples are s32 / s64 (indexed from tile_begin).
// Adds the fixed-point partial SSE of each candidate into acc[cand] (shared).
// Items (tile t, group g) = it, it = t * G + g (t counted from tile_begin),
// go to warps round-robin; for
// the default tier each warp computes the tile anchors of its next IPB items
// itself into its own slice of `anc` (IPB * CGV entries per warp), so no
// CTA-wide barrier separates anchors from evaluation. Each warp then calls
// hook(warp) (work for warps that finish early); ends with __syncthreads().
struct NoHook {
  __device__ void operator()(int) const {}
};
template <int TIER, int CGV, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC, class Hook = NoHook>
__device__ void eval_range(const BlockArgs& b, int64_t tile_begin, int item_lo, int item_hi, const float* s32,
                           const double* s64, const unsigned char* cdata, const float* negA, const int* kexp,
                           const unsigned char* cub, int ncand, int npad, uint4* anc, unsigned long long* acc,
                           const Hook& hook = Hook()) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int G = npad / CGV;
  const int nitems = item_hi;
  const dfloat t0d = df_from_double(b.t0), hd = df_from_double(b.h);
  const float t0f = __double2float_rn(b.t0), hf = __double2float_rn(b.h);
  constexpr int AW = anchor_words(MODEL);
  uint4* anc_w = anc + warp * (IPB * CGV * AW);
  constexpr int LPC = 32 / CGV;  // lanes holding each candidate's warp sum

  for (int base = item_lo + warp; base < nitems; base += nw * IPB) {
    if constexpr (MODEL == MODEL_FULL && TIER == TIER_F64) {
      for (int q = lane; q < IPB * CGV; q += 32) {
        const int k = q / CGV, c = q - k * CGV;
        const int it = base + k * nw;
        uint4 av[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        if (it < nitems) {
          const int t = it / G, cand = (it - t * G) * CGV + c;
          if (cand < ncand) {
            const unsigned char* cd = cdata + cand * CAND_BYTES_FULL;
            const u128* e = reinterpret_cast<const u128*>(cd);
            const u128 ev[5] = {e[0], e[1], e[2], e[3], e[4]};
            const float* am = reinterpret_cast<const float*>(cd + 80);
            make_anchor_full(ev, (uint64_t)(tile_begin + t) * (uint64_t)L + L / 2, am[0], am[1], av);
          }
        }
        anc_w[2 * q] = av[0];
        anc_w[2 * q + 1] = av[1];
      }
      __syncwarp();
    } else if (TIER == TIER_F64) {
      for (int q = lane; q < IPB * CGV; q += 32) {
        const int k = q / CGV, c = q - k * CGV;
        const int it = base + k * nw;
        uint4 av = make_uint4(0, 0, 0, 0);
        if (it < nitems) {
          const int t = it / G, cand = (it - t * G) * CGV + c;
          if (cand < ncand) {
            const u128* e = reinterpret_cast<const u128*>(cdata + cand * CAND_BYTES);
            Poly P;
            P.e[0] = e[0];
            P.e[1] = e[1];
            P.e[2] = e[2];
            P.e[3] = e[3];
            av = make_anchor(P, (uint64_t)(tile_begin + t) * (uint64_t)L);
          }
        }
        anc_w[q] = av;
      }
      __syncwarp();
    }
#pragma unroll 1
    for (int k = 0; k < IPB; ++k) {
      const int it = base + k * nw;
      if (it >= nitems) break;
      const int t = it / G, g = it - t * G;
      const int64_t tstart = (tile_begin + t) * (int64_t)L;
      const int64_t rem = b.n - tstart;
      const int nvalid = rem < L ? (int)rem : L;
      const int64_t soff = (int64_t)t * L + lane * M;
      const int cand = g * CGV + lane / LPC;
      const bool owner = (lane & (LPC - 1)) == 0 && cand < ncand;
      if (TIER == TIER_PLAIN) {
        double s[M];
#pragma unroll
        for (int m = 0; m < M; m += 2) {
          const double2 v = *reinterpret_cast<const double2*>(s64 + soff + m);
          s[m] = v.x;
          s[m + 1] = v.y;
        }
        double accv[CGV];
        const unsigned char* cdp = cdata + g * CGV * cand_bytes(MODEL);
        if (nvalid == L) item_plain<CGV, false, OBJ, MODEL>(s, cdp, lane, nvalid, tstart, b, accv);
        else item_plain<CGV, true, OBJ, MODEL>(s, cdp, lane, nvalid, tstart, b, accv);
        const double z = warp_reduce_scatter<CGV>(accv, lane);
        if (owner) {
          const long long v = __double2ll_rn(z * __longlong_as_double((long long)(1023 + kexp[cand]) << 52));
          atomicAdd(&acc[cand], (unsigned long long)v);
        }
      } else {
        float s[M];
#pragma unroll
        for (int m = 0; m < M; m += 4) {
          const float4 v = *reinterpret_cast<const float4*>(s32 + soff + m);
          s[m] = v.x;
          s[m + 1] = v.y;
          s[m + 2] = v.z;
          s[m + 3] = v.w;
        }
        float accv[CGV];
        const float* nA = negA + g * CGV;
        const unsigned char* cd = cdata + g * CGV * cand_bytes(MODEL);
        if constexpr (MODEL == MODEL_FULL && TIER == TIER_F64) {
          const uint4* anc_i = anc_w + k * CGV * 2;
          if (nvalid == L) {
            if (any_flag<CGV>(cub + g * CGV)) item_full_mixed<CGV>(s, anc_i, cub + g * CGV, lane, accv);
            else item_full_fold<CGV>(s, anc_i, lane, accv);
          } else {
            item_full_masked<CGV>(s, anc_i, lane, nvalid, accv);
          }
        } else if (TIER == TIER_F64) {
          const uint4* anc_i = anc_w + k * CGV;
          if (nvalid == L) {
            if (any_flag<CGV>(cub + g * CGV)) item_f64_mixed<CGV, OBJ>(s, anc_i, nA, cub + g * CGV, lane, accv);
            else item_f64_fold<CGV, OBJ>(s, anc_i, nA, lane, accv);
          } else {
            item_f64<CGV, true, OBJ>(s, anc_i, nA, lane, nvalid, accv);
          }
        } else if (TIER == TIER_DF32) {
          if (nvalid == L) item_df32<CGV, false, OBJ, MODEL>(s, cd, nA, lane, nvalid, tstart, t0d, hd, accv);
          else item_df32<CGV, true, OBJ, MODEL>(s, cd, nA, lane, nvalid, tstart, t0d, hd, accv);
        } else {
          if (nvalid == L) item_f32<CGV, false, OBJ, MODEL>(s, cd, nA, lane, nvalid, tstart, t0f, hf, accv);
          else item_f32<CGV, true, OBJ, MODEL>(s, cd, nA, lane, nvalid, tstart, t0f, hf, accv);
        }
        const float z = warp_reduce_scatter<CGV>(accv, lane);
        if (owner) {
          const long long v = __float2ll_rn(z * exp2_int_f(kexp[cand]));
          atomicAdd(&acc[cand], (unsigned long long)v);
        }
      }
    }
    __syncwarp();
  }
  hook(warp);
  __syncthreads();
}

// Stage tiles [tb, tb + nt) of the block into shared memory and convert them.
// Returns false (and sets *err) if the bulk copy did not complete in time.
// extra_tx: see bulk_stage (0 except in the test of the wait's limit).
template <int TIER>
__device__ bool stage_tiles(const BlockArgs& b, int64_t tb, int nt, void* raw, float* s32, double* s64,
                            uint64_t* mbar, uint64_t timeout_ns, int* err, uint32_t extra_tx = 0) {
  const uint32_t bytes = (uint32_t)nt * (uint32_t)L * (uint32_t)b.esize;
  const char* src = reinterpret_cast<const char*>(b.samples) + tb * (int64_t)L * b.esize;
  if (!bulk_stage(raw, src, bytes, mbar, timeout_ns, extra_tx)) {
    if (threadIdx.x == 0) atomicExch(err, DEV_TIMEOUT);
    return false;
  }
  const int cnt = nt * L;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const double v = load_physical(raw, b.dtype, i, b.scale);
    if (tier_uses_f64_samples(TIER)) s64[i] = v;
    else s32[i] = __double2float_rn(v);
  }
  __syncthreads();
  return true;
}

// Shared-memory carve-up common to both kernels.
struct SmemLayout {
  size_t off_mbar, off_cdata, off_negA, off_kexp, off_cub, off_acc, off_draw, off_anc, off_samp, off_raw, off_pop,
      off_u2, off_cdata2, off_negA2, off_kexp2, off_cub2, off_win, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// npad: padded candidates; tmax: max tiles per CTA; cgv: candidates per item;
// pop: population slots (0 for the objective kernel); nthreads: CTA size.
// model: MODEL_CUBIC or MODEL_FULL (wider population rows, candidate data and anchors).
// With pop > 0 (the DE): two generations' draws, a replacement flag per
// individual and, with `ahead_set`, a second set of trials and set-up (the
// next generation's, built ahead); the current generation's set keeps fixed
// offsets ahead of them.
__host__ __device__ inline SmemLayout smem_layout(int tier, int npad, int tmax, int cgv, int esize, int pop,
                                                  int nthreads, int model = MODEL_CUBIC, bool ahead_set = true) {
  SmemLayout s;
  size_t o = 0;
  const size_t ahead = (pop && ahead_set) ? 1 : 0;
  s.off_mbar = o;
  o += 16;
  s.off_pop = o;
  o += align_up((size_t)pop * (2 * model_dim(model) + 1) * sizeof(double), 16);
  s.off_cdata = o;
  o += (size_t)npad * cand_bytes(model);
  s.off_negA = o;
  o += align_up((size_t)npad * sizeof(float), 16);
  s.off_kexp = o;
  o += align_up((size_t)npad * sizeof(int), 16);
  s.off_cub = o;
  o += align_up((size_t)npad, 16);
  s.off_acc = o;
  o += align_up((size_t)npad * sizeof(unsigned long long), 16);
  s.off_draw = o;
  // rpack, take and model_dim jitter words per individual, for two generations
  o += align_up((size_t)(pop ? 2 * (2 + model_dim(model)) * npad : 0) * sizeof(uint32_t), 16);
  s.off_u2 = o;
  o += ahead * align_up((size_t)pop * model_dim(model) * sizeof(double), 16);
  s.off_cdata2 = o;
  o += ahead * (size_t)npad * cand_bytes(model);
  s.off_negA2 = o;
  o += ahead * align_up((size_t)npad * sizeof(float), 16);
  s.off_kexp2 = o;
  o += ahead * align_up((size_t)npad * sizeof(int), 16);
  s.off_cub2 = o;
  o += ahead * align_up((size_t)npad, 16);
  s.off_win = o;  // the replacement flags: every DE launch
  o += (pop ? 1 : 0) * align_up((size_t)npad, 16);
  s.off_anc = o;
  o += (tier == TIER_F64) ? (size_t)(nthreads / 32) * IPB * cgv * anchor_words(model) * sizeof(uint4) : 0;
  s.off_samp = o;
  o += align_up((size_t)tmax * L * (tier_uses_f64_samples(tier) ? 8 : 4), 128);
  s.off_raw = o;
  o += align_up((size_t)tmax * L * esize, 128);
  s.total = o;
  return s;
}

// ---------------------------------------------------------------------------

static __global__ void k_absmax(const void* samples, int64_t n, int dtype, unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(load_physical(samples, dtype, i, 1.0)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

struct ObjArgs {
  BlockArgs b;
  const double* cands;
  int ncand;
  int tpc;          // tiles per CTA (grid.x)
  int cpc;          // candidates per CTA, multiple of the item width (grid.y)
  unsigned long long* acc;  // [ncand], zeroed by the caller
  int* err;
  uint64_t timeout_ns;
  uint32_t extra_tx;        // 0, or the bytes a test of the staging wait adds (bulk_stage)
};

template <int TIER, int CGV, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
__global__ void __launch_bounds__(NT_OBJ, OBJ_CTAS) k_objective(ObjArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t tb = (int64_t)blockIdx.x * a.tpc;
  const int nt = (int)min((int64_t)a.tpc, a.b.ntiles - tb);
  const int cb = blockIdx.y * a.cpc;
  const int nc = min(a.cpc, a.ncand - cb);
  if (nt <= 0 || nc <= 0) return;
  const int npad = (nc + CGV - 1) / CGV * CGV;
  const SmemLayout S = smem_layout(TIER, npad, a.tpc, CGV, a.b.esize, 0, NT_OBJ, MODEL);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S.off_mbar);
  unsigned char* cdata = smem + S.off_cdata;
  float* negA = reinterpret_cast<float*>(smem + S.off_negA);
  int* kexp = reinterpret_cast<int*>(smem + S.off_kexp);
  unsigned char* cub = smem + S.off_cub;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem + S.off_acc);
  uint4* anc = reinterpret_cast<uint4*>(smem + S.off_anc);
  float* s32 = reinterpret_cast<float*>(smem + S.off_samp);
  double* s64 = reinterpret_cast<double*>(smem + S.off_samp);
  void* raw = smem + S.off_raw;

  const int tid = threadIdx.x;
  if (tid < npad) acc[tid] = 0ull;
  prep_all<TIER, OBJ, MODEL>(a.cands + (int64_t)cb * model_dim(MODEL), nc, npad, a.b, cdata, negA, kexp, cub,
                             OBJ == OBJ_COR ? COR_BITS_OBJ : SSE_BITS_OBJ);
  if (!stage_tiles<TIER>(a.b, tb, nt, raw, s32, s64, mbar, a.timeout_ns, a.err, a.extra_tx)) return;
  eval_range<TIER, CGV, OBJ, MODEL>(a.b, tb, 0, nt * (npad / CGV), s32, s64, cdata, negA, kexp, cub, nc, npad, anc,
                                    acc);
  if (tid < nc) atomicAdd(&a.acc[cb + tid], acc[tid]);
}

// The objective value of each candidate from its fixed-point sum: the SSE,
// or for OBJ_COR F_cor from S = sum s_i cos(phi_i) and the candidate's A.
// model MODEL_FULL: rows of 7 parameters, the full model's exponent (t0, h
// give its amplitude terms).
static __global__ void k_finalize(const double* cands, int ncand, const unsigned long long* acc, int64_t n, float smax_f,
                                  double* sse, int obj, int model, double t0, double h) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand) return;
  if (model == MODEL_FULL) {
    const AmpTerms am = full_amp(cands + (int64_t)c * DF, t0, h);
    sse[c] = fixed_to_double(acc[c], full_scale_exp(am, n, smax_f, SSE_BITS_OBJ));
    return;
  }
  const double A = cands[(int64_t)c * D];
  if (obj == OBJ_COR) {
    sse[c] = cor_objective_value(A, signed_fixed_to_double((long long)acc[c], cor_scale_exp(n, smax_f, COR_BITS_OBJ)));
  } else {
    sse[c] = fixed_to_double(acc[c], sse_scale_exp(n, smax_f, fabsf(__double2float_rn(A)), SSE_BITS_OBJ));
  }
}

// One block's DE problem (device-side descriptor).
struct DeBlockDesc {
  BlockArgs b;
  DeControls dc;
  int np, gens;
  int cg;            // candidates per work item for this block (16, 8 or 4)
  double* out;       // [dim + 1] device: best params + SSE
  double* pop_out;   // [np * dim] device or nullptr
  double* fit_out;   // [np] device or nullptr
};

// A persistent DE launch: `ngroups` groups of `k` co-resident CTAs; group q
// solves blocks sched[sched_off[q] .. sched_off[q+1]) in order.
struct DeLaunch {
  const DeBlockDesc* blocks;
  const int* sched;
  const int* sched_off;
  int ngroups, k;
  int sc_tiles;              // tiles staged per CTA at a time (shared-memory budget)
  int esize_max;             // largest sample size in the launch (shared-memory layout)
  unsigned long long* ring;  // [ngroups][RING_SLOTS][NP_MAX][RING_STRIDE], zeroed by the caller
  int* err;                  // zeroed by the caller
  uint64_t timeout_ns;
  int obj;                   // OBJ_CHI2 or OBJ_COR (the kernel instantiation launched)
  uint32_t extra_tx;         // 0, or the bytes a test of the staging wait adds (bulk_stage)
  int ahead;                 // the second trial set is laid out (every block of the launch is resident)
};

// One generation's draws: packed indices, crossover mask, model_dim jitter
// words per individual.
struct Draws {
  uint32_t *drp, *drt, *drj;
};

struct DeSmem {
  uint64_t* mbar;
  double *x, *u, *fx;
  unsigned char* cdata;
  float* negA;
  int* kexp;
  unsigned char* cub;
  unsigned long long* acc;
  // the next generation's trials and set-up, when built ahead (AheadHook)
  double* u2;
  unsigned char* cdata2;
  float* negA2;
  int* kexp2;
  unsigned char* cub2;
  unsigned char* win;   // per individual: replaced at the last selection
  Draws dr0, dr1;       // generation g's draws are set g & 1 (picked by value, off the evaluation)
  __device__ __forceinline__ Draws draws(int g) const { return (g & 1) ? dr1 : dr0; }
  uint4* anc;
  float* s32;
  double* s64;
  void* raw;
};

// The lowest-index minimum of fx[0 .. np) (the order of dkey), found by a
// whole warp: each lane takes every 32nd individual in ascending order, then
// a shuffle reduction keeps the smaller key, or on equal keys the smaller
// index, so the result is the first minimum a sequential scan would find.
// Every lane of the warp must call it.
__device__ __forceinline__ int lowest_minimum_warp(const double* fx, int np, int lane) {
  long long bk = LLONG_MAX;
  int bi = INT_MAX;
  for (int i = lane; i < np; i += 32) {
    const long long ki = dkey(fx[i]);
    if (ki < bk) {
      bk = ki;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ok < bk || (ok == bk && oi < bi)) {
      bk = ok;
      bi = oi;
    }
  }
  return bi;
}

// Trial components of the generation from population x and draws dr into u:
// with a list, every component of the trials list[0 .. nlist), otherwise of
// all np trials; one (individual, component) per thread, from `first` in
// steps of `stride`. DE_BEST1_JITTER mutates from the previous generation's
// lowest-index minimum (of fx), which every warp finds itself
// (lowest_minimum_warp: broadcast reads of the fitnesses, no extra CTA
// barrier); its callers are whole warps.
template <int STRAT, int DIM = D>
__device__ __forceinline__ void mutate_all(const DeControls& dc, const double* x, const double* fx, double* u,
                                           const Draws& dr, int np, int npad, int first, int stride,
                                           const unsigned char* list = nullptr, int nlist = 0) {
  int best = 0;
  if (STRAT == DE_BEST1_JITTER) best = lowest_minimum_warp(fx, np, threadIdx.x & 31);
  const int m = list ? nlist : npad;
  for (int t = first; t < DIM * m; t += stride) {
    const int j = t / m, i = t - j * m;
    const int c = list ? (int)list[i] : i;
    if (c < np)
      u[c * DIM + j] = de_component<STRAT, DIM>(dc, x, c, j, dr.drp[c], dr.drt[c], best, dr.drj + c * DIM);
  }
}

template <int DIM = D>
__device__ __forceinline__ void mutate_any(int strat, const DeControls& dc, const double* x, const double* fx,
                                           double* u, const Draws& dr, int np, int npad, int first, int stride,
                                           const unsigned char* list = nullptr, int nlist = 0) {
  if (strat == DE_BEST1_JITTER)
    mutate_all<DE_BEST1_JITTER, DIM>(dc, x, fx, u, dr, np, npad, first, stride, list, nlist);
  else if (strat == DE_EITHER_OR)
    mutate_all<DE_EITHER_OR, DIM>(dc, x, fx, u, dr, np, npad, first, stride, list, nlist);
  else mutate_all<DE_RAND1_BIN, DIM>(dc, x, fx, u, dr, np, npad, first, stride, list, nlist);
}

// Generation `gen`'s draws for individual c into dr.
template <int DIM = D>
__device__ __forceinline__ void draw_any(int strat, const DeControls& dc, int np, int c, uint32_t gen,
                                         const Draws& dr) {
  if (strat == DE_BEST1_JITTER)
    de_draws<DE_BEST1_JITTER, DIM>(dc, np, c, gen, &dr.drp[c], &dr.drt[c], dr.drj + c * DIM);
  else if (strat == DE_EITHER_OR)
    de_draws<DE_EITHER_OR, DIM>(dc, np, c, gen, &dr.drp[c], &dr.drt[c], dr.drj + c * DIM);
  else de_draws<DE_RAND1_BIN, DIM>(dc, np, c, gen, &dr.drp[c], &dr.drt[c], dr.drj + c * DIM);
}

__device__ __forceinline__ void bar_sync_named(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Warps that hold one item fewer than warp 0 leave the evaluation early; while
// the others finish, warps first_warp .. end build the next generation's
// trials (its draws are ready) and their set-up, into the second set, from the
// current population, as if the coming selection replaced no individual.
// After the selection the trials that read a replaced individual (their own
// parent or one of their three donors) are rebuilt; every other trial has
// exactly the inputs, and so the bits, that the generation would have
// computed after the selection. Named barrier 1 orders the trials before
// their set-up among these warps only. Not for DE_BEST1_JITTER, whose base
// vector is the selection's best.
template <int DIM, int TIER, int OBJ, int MODEL>
struct AheadHook {
  const DeControls* dc;
  const BlockArgs* b;
  const DeSmem* sm;
  Draws dr;
  int strat, np, npad, first_warp, kbits;
  __device__ void operator()(int warp) const {
    if (warp < first_warp) return;
    const int nthr = (int)blockDim.x - first_warp * 32, q = (int)threadIdx.x - first_warp * 32;
    if (strat == DE_EITHER_OR)
      mutate_all<DE_EITHER_OR, DIM>(*dc, sm->x, nullptr, sm->u2, dr, np, npad, q, nthr);
    else mutate_all<DE_RAND1_BIN, DIM>(*dc, sm->x, nullptr, sm->u2, dr, np, npad, q, nthr);
    bar_sync_named(1, nthr);
    prep_range<TIER, OBJ, MODEL>(sm->u2, np, npad, *b, sm->cdata2, sm->negA2, sm->kexp2, sm->cub2, kbits, q, nthr);
  }
};

// Fewest early warps worth building the next generation ahead, and most
// individuals the last selection may have replaced for it (acceptance is high
// early in a fit, when most trials would be rebuilt anyway; on the 400K block
// a limit of 1 beat 0, 2, 4, 8 and 16).
constexpr int AHEAD_MIN_WARPS = 4;
constexpr int AHEAD_MAX_REPLACED = 1;

// After a selection that replaced individuals, rebuild in the current buffers
// the trials built ahead that read one of them (their own parent or a
// donor): every warp finds the stale set itself (a trial and its three donor
// flags per lane, a ballot per 32 trials), and warp w rebuilds the stale
// trials of rank w, w + nw, ...: its lanes make the trial's components, then
// its set-up tasks. No barrier: the caller's next one orders the results.
template <int DIM, int TIER, int OBJ, int MODEL>
__device__ __forceinline__ void rebuild_stale(int strat, const DeControls& dc, const BlockArgs& b, const DeSmem& sm,
                                              const Draws& dr, int np, int npad, int kbits) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int rank = 0;
  for (int c0 = 0; c0 < np; c0 += 32) {
    const int c = c0 + lane;
    bool stale = false;
    if (c < np) {
      const uint32_t rp = dr.drp[c];
      stale = (sm.win[c] | sm.win[rp & 0xff] | sm.win[(rp >> 8) & 0xff] | sm.win[(rp >> 16) & 0xff]) != 0;
    }
    unsigned m = __ballot_sync(0xffffffffu, stale);
    while (m) {
      const int t = c0 + __ffs(m) - 1;
      m &= m - 1u;
      if (rank++ % nw != warp) continue;
      if (lane < DIM) {
        sm.u[t * DIM + lane] =
            strat == DE_EITHER_OR
                ? de_component<DE_EITHER_OR, DIM>(dc, sm.x, t, lane, dr.drp[t], dr.drt[t], 0, dr.drj + t * DIM)
                : de_component<DE_RAND1_BIN, DIM>(dc, sm.x, t, lane, dr.drp[t], dr.drt[t], 0, dr.drj + t * DIM);
      }
      __syncwarp();
      prep_range<TIER, OBJ, MODEL>(sm.u, np, npad, b, sm.cdata, sm.negA, sm.kexp, sm.cub, kbits, lane, 32, nullptr,
                                   0, t);
      __syncwarp();
    }
  }
}

// During the exchange wait (this generation's evaluation done), threads
// `first` in steps of `stride` move the set-up built ahead into the current
// buffers: every candidate's row, -A and flag, and the exponents of the
// padding candidates; each of the first np candidates' poller moves its
// exponent and trial row itself once it has used them.
template <int MODEL>
__device__ __forceinline__ void take_ahead_setup(const DeSmem& sm, int np, int npad, int first, int stride) {
  constexpr int CB = cand_bytes(MODEL);
  static_assert(CB % 16 == 0, "candidate rows copy as 16-byte words");
  const uint4* src = reinterpret_cast<const uint4*>(sm.cdata2);
  uint4* dst = reinterpret_cast<uint4*>(sm.cdata);
  for (int i = first; i < npad * (CB / 16); i += stride) dst[i] = src[i];
  for (int i = first; i < npad; i += stride) {
    sm.negA[i] = sm.negA2[i];
    sm.cub[i] = sm.cub2[i];
    if (i >= np) sm.kexp[i] = sm.kexp2[i];
  }
}

// DE (the block's strategy) on one block by `k` CTAs (this one is `rank`). Every CTA holds
// the whole population and generates every trial itself (identical Philox
// draws, identical FP64 arithmetic), so the only exchange is each trial's SSE:
// every CTA adds (partial << 8) | 1 to the trial's 64-bit word of the group's
// RING_SLOTS-deep ring, whose low byte counts arrivals; a word whose low byte equals k
// holds the complete fixed-point sum, and one acquire load per candidate
// replaces a barrier, a fence and a separate read. `gg` counts the group's
// generations across blocks so the ring discipline continues from block to
// block. Generation g's draws are made during generation g - 2's exchange
// wait; its trials and set-up are built during generation g - 1's evaluation
// where the CTA has early warps and the last selection replaced few
// individuals (AheadHook), else after the selection. s_nrep[2] counts each
// generation's replacements. Returns false if a bounded wait expired or
// another CTA failed.
// MODEL_FULL: the full model's 7 parameters (chi-square).
// SK: the launch's strategy when fixed at compile time, -1 to read it from the block.
template <int TIER, int CGV, int OBJ, int MODEL = MODEL_CUBIC, int SK = -1, bool STREAM = true>
__device__ bool de_block(const DeBlockDesc& d, int rank, int k, unsigned long long* ring, unsigned long long& gg,
                         const DeSmem& sm, const DeLaunch& a, int* s_abort, int* s_nrep) {
  constexpr int DIM = model_dim(MODEL);
  constexpr int KBITS = OBJ == OBJ_COR ? COR_BITS_DE : SSE_BITS_DE;
  const int strat = SK >= 0 ? SK : d.dc.strategy;
  const int tid = threadIdx.x, nw = (int)(blockDim.x >> 5);
  const int np = d.np, npad = (d.np + CGV - 1) / CGV * CGV;
  const BlockArgs& b = d.b;
  // this CTA's share of the block's items (tile, candidate group), in tile
  // order: item-exact, so the CTAs' shares differ by at most one item; it
  // spans the staged tiles [tb, tb + nt), items [ilo, ihi) counted from tb
  const int G = npad / CGV;
  const int64_t nitems = b.ntiles * G;
  const int64_t it0 = (int64_t)rank * nitems / k, it1 = (int64_t)(rank + 1) * nitems / k;
  const int64_t tb = it0 / G;
  const int nt = it1 > it0 ? (int)((it1 - 1) / G - tb + 1) : 0;
  const int ilo = (int)(it0 - tb * G), ihi = (int)(it1 - tb * G);
  const bool resident = nt <= a.sc_tiles;
  const unsigned long long arrived = (unsigned long long)(k & 0xff);
  // items go to warps round-robin, so warps rem .. nw - 1 hold one item fewer
  // than warp 0 (none when rem = 0)
  const int rem = (ihi - ilo) % nw;
  const int first_early =
      (a.ahead && resident && strat != DE_BEST1_JITTER && rem > 0 && nw - rem >= AHEAD_MIN_WARPS) ? rem : -1;
  if (resident && nt > 0 &&
      !stage_tiles<TIER>(b, tb, nt, sm.raw, sm.s32, sm.s64, sm.mbar, a.timeout_ns, a.err, a.extra_tx))
    return false;

  bool ahead = false;  // this generation's trials and set-up were built during the last evaluation
  for (int gen = 0; gen <= d.gens; ++gen, ++gg) {
    unsigned long long* slot = ring + (gg % RING_SLOTS) * (NP_MAX * RING_STRIDE);
    const Draws dr = sm.draws(gen);
    // replacements at the last selection (all of generation 0's)
    const int nrep = gen > 0 ? s_nrep[(gen - 1) & 1] : np;
    if (tid == 0) s_nrep[gen & 1] = 0;
    // trials u of this generation (the initial population at gen 0) and their set-up
    if (gen == 0) {
      if (tid < np) de_init<DIM>(d.dc, tid, sm.u + tid * DIM);
      if (tid < npad) sm.acc[tid] = 0ull;
      __syncthreads();
      prep_all<TIER, OBJ, MODEL>(sm.u, np, npad, b, sm.cdata, sm.negA, sm.kexp, sm.cub, KBITS);
    } else if (ahead) {
      // the trials and set-up built ahead are in place (moved during the last
      // exchange); those that read an individual the selection replaced are rebuilt
      if (nrep > 0) {
        rebuild_stale<DIM, TIER, OBJ, MODEL>(strat, d.dc, b, sm, dr, np, npad, KBITS);
        __syncthreads();
      }
    } else {
      mutate_any<DIM>(strat, d.dc, sm.x, sm.fx, sm.u, dr, np, npad, tid, blockDim.x);
      __syncthreads();
      prep_all<TIER, OBJ, MODEL>(sm.u, np, npad, b, sm.cdata, sm.negA, sm.kexp, sm.cub, KBITS);
    }
    const bool build_next = first_early >= 0 && gen >= 1 && gen < d.gens && nrep <= AHEAD_MAX_REPLACED;
    if (build_next) {
      const AheadHook<DIM, TIER, OBJ, MODEL> hook{&d.dc, &b, &sm, sm.draws(gen + 1), strat, np, npad, first_early, KBITS};
      eval_range<TIER, CGV, OBJ, MODEL>(b, tb, ilo, ihi, sm.s32, sm.s64, sm.cdata, sm.negA, sm.kexp, sm.cub, np, npad,
                                        sm.anc, sm.acc, hook);
    } else if (resident) {
      eval_range<TIER, CGV, OBJ, MODEL>(b, tb, ilo, ihi, sm.s32, sm.s64, sm.cdata, sm.negA, sm.kexp, sm.cub, np, npad,
                                        sm.anc, sm.acc);
    } else if constexpr (STREAM) {
      for (int c0 = 0; c0 < nt; c0 += a.sc_tiles) {
        const int cn = min(a.sc_tiles, nt - c0);
        const int lo = max(ilo, c0 * G) - c0 * G, hi = min(ihi, (c0 + cn) * G) - c0 * G;
        if (!stage_tiles<TIER>(b, tb + c0, cn, sm.raw, sm.s32, sm.s64, sm.mbar, a.timeout_ns, a.err, a.extra_tx))
          return false;
        eval_range<TIER, CGV, OBJ, MODEL>(b, tb + c0, lo, hi, sm.s32, sm.s64, sm.cdata, sm.negA, sm.kexp, sm.cub, np,
                                          npad, sm.anc, sm.acc);
      }
    } else {
      // compiled for resident tiles only: the launcher picks this kernel when
      // every CTA's share fits, so this is a launcher error, reported
      atomicExch(a.err, DEV_LAYOUT);
      return false;
    }
    ahead = build_next;
    if (tid < np) {
      unsigned long long* w = slot + tid * RING_STRIDE;
      const unsigned long long contrib = (sm.acc[tid] << 8) | 1ull;
      sm.acc[tid] = 0ull;  // for the next generation (the closing barrier orders it)
      atomicAdd(w, contrib);
      // wait for every CTA's contribution to this candidate, then select
      const uint64_t t_start = globaltimer_ns();
      unsigned long long v;
      int spins = 0;
      while (((v = ld_acquire_u64(w)) & 0xffull) != arrived) {
        if ((++spins & 63) == 0) {
          if (ld_volatile_i32(a.err) != DEV_OK) {
            *s_abort = 1;
            break;
          }
          if (globaltimer_ns() - t_start > a.timeout_ns) {
            atomicExch(a.err, DEV_TIMEOUT);
            *s_abort = 1;
            break;
          }
        }
      }
      // the words' sums are signed for OBJ_COR (two's complement adds); the low
      // byte counts arrivals either way
      // OBJ_COR ranks by -cor (F_cor = 1/(atan(cor) + pi/2) decreases strictly
      // with cor), so no FP64 arctangent sits on the generation's critical
      // path; F_cor is formed once for the outputs. dkey orders signed doubles.
      const double f = OBJ == OBJ_COR
                           ? -(sm.u[tid * DIM] * signed_fixed_to_double((long long)v >> 8, sm.kexp[tid]))
                           : fixed_to_double(v >> 8, sm.kexp[tid]);
      const bool replace = gen == 0 || dkey(f) <= dkey(sm.fx[tid]);
      if (replace) {
        sm.fx[tid] = f;
#pragma unroll
        for (int j = 0; j < DIM; ++j) sm.x[tid * DIM + j] = sm.u[tid * DIM + j];
        atomicAdd(&s_nrep[gen & 1], 1);
      }
      sm.win[tid] = replace ? 1 : 0;
      if (build_next) {
        // the next generation's trial and exponent, built ahead, now that this one's are used
#pragma unroll
        for (int j = 0; j < DIM; ++j) sm.u[tid * DIM + j] = sm.u2[tid * DIM + j];
        sm.kexp[tid] = sm.kexp2[tid];
      }
    } else if (rank == 0 && tid >= 2 * NP_MAX && tid < 3 * NP_MAX) {
      // Slot gg + 2 was last used at generation gg - 2, whose words every CTA
      // read before contributing to gg - 1, which rank 0 has seen complete;
      // rank 0 clears it now, off the exchange's critical path, and the fence
      // puts the clear before the closing barrier, so before rank 0's
      // contributions to gg + 1, which every CTA observes before it
      // contributes to gg + 2. (Every word of the slot: the group's next block
      // may have a larger population.)
      ring[((gg + 2) % RING_SLOTS) * (NP_MAX * RING_STRIDE) + (tid - 2 * NP_MAX) * RING_STRIDE] = 0ull;
      __threadfence();
    } else if (tid >= NP_MAX && tid < NP_MAX + np) {
      // draws do not depend on selection: generation gen + 2's are made during
      // this wait, into the set generation gen has finished with
      if (gen + 2 <= d.gens) draw_any<DIM>(strat, d.dc, np, tid - NP_MAX, (uint32_t)(gen + 2), dr);
    } else if (gen == 0 && d.gens >= 1 && tid >= 3 * NP_MAX && tid < 3 * NP_MAX + np) {
      draw_any<DIM>(strat, d.dc, np, tid - 3 * NP_MAX, 1u, sm.dr1);
    } else if (build_next && tid >= 3 * NP_MAX) {
      take_ahead_setup<MODEL>(sm, np, npad, tid - 3 * NP_MAX, (int)blockDim.x - 3 * NP_MAX);
    }
    __syncthreads();
    if (*s_abort) return false;
  }
  if (rank == 0) {
    if (tid == 0) {
      int best = 0;
      for (int i = 1; i < np; ++i)
        if (dkey(sm.fx[i]) < dkey(sm.fx[best])) best = i;
      for (int j = 0; j < DIM; ++j) d.out[j] = sm.x[best * DIM + j];
      d.out[DIM] = OBJ == OBJ_COR ? cor_objective_value(1.0, -sm.fx[best]) : sm.fx[best];
    }
    if (d.pop_out)
      for (int i = tid; i < np * DIM; i += blockDim.x) d.pop_out[i] = sm.x[i];
    if (d.fit_out)
      for (int i = tid; i < np; i += blockDim.x)
        d.fit_out[i] = OBJ == OBJ_COR ? cor_objective_value(1.0, -sm.fx[i]) : sm.fx[i];
  }
  __syncthreads();
  return true;
}

// Persistent DE launch over groups of blocks (one block: one group of all CTAs).
// Launched cooperatively: the k CTAs of a group wait on one another. OBJ
// selects the objective every block of the launch minimises; SK, when not -1,
// the DE strategy of all its blocks (each strategy's kernel then holds only
// its own trial code). CGK = 16, with SK: every block of the launch evaluates
// 16-candidate items on resident tiles, so the kernel holds that one form of
// the evaluation (no other item width, no streaming of tiles).
template <int TIER, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC, int SK = -1, int CGK = 0>
__global__ void __launch_bounds__(NT, 1) k_de(DeLaunch a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int DIM = model_dim(MODEL);
  const SmemLayout S = smem_layout(TIER, NP_MAX, a.sc_tiles, 16, a.esize_max, NP_MAX, NT, MODEL, a.ahead != 0);
  DeSmem sm;
  sm.mbar = reinterpret_cast<uint64_t*>(smem + S.off_mbar);
  sm.x = reinterpret_cast<double*>(smem + S.off_pop);
  sm.u = sm.x + NP_MAX * DIM;
  sm.fx = sm.u + NP_MAX * DIM;
  sm.cdata = smem + S.off_cdata;
  sm.negA = reinterpret_cast<float*>(smem + S.off_negA);
  sm.kexp = reinterpret_cast<int*>(smem + S.off_kexp);
  sm.cub = smem + S.off_cub;
  sm.acc = reinterpret_cast<unsigned long long*>(smem + S.off_acc);
  sm.u2 = reinterpret_cast<double*>(smem + S.off_u2);
  sm.cdata2 = smem + S.off_cdata2;
  sm.negA2 = reinterpret_cast<float*>(smem + S.off_negA2);
  sm.kexp2 = reinterpret_cast<int*>(smem + S.off_kexp2);
  sm.cub2 = smem + S.off_cub2;
  sm.win = smem + S.off_win;
  sm.dr0.drp = reinterpret_cast<uint32_t*>(smem + S.off_draw);
  sm.dr0.drt = sm.dr0.drp + NP_MAX;
  sm.dr0.drj = sm.dr0.drp + 2 * NP_MAX;
  sm.dr1.drp = sm.dr0.drp + (2 + DIM) * NP_MAX;
  sm.dr1.drt = sm.dr1.drp + NP_MAX;
  sm.dr1.drj = sm.dr1.drp + 2 * NP_MAX;
  sm.anc = reinterpret_cast<uint4*>(smem + S.off_anc);
  sm.s32 = reinterpret_cast<float*>(smem + S.off_samp);
  sm.s64 = reinterpret_cast<double*>(smem + S.off_samp);
  sm.raw = smem + S.off_raw;
  __shared__ int s_abort, s_nrep[2];
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();

  const int q = blockIdx.x / a.k, rank = blockIdx.x - q * a.k;
  if (q >= a.ngroups) return;
  unsigned long long* ring = a.ring + (size_t)q * RING_SLOTS * NP_MAX * RING_STRIDE;
  unsigned long long gg = 0;
  __shared__ DeBlockDesc s_desc;
  for (int e = a.sched_off[q]; e < a.sched_off[q + 1]; ++e) {
    // the block's descriptor lives in shared memory while it is solved
    if (threadIdx.x == 0) s_desc = a.blocks[a.sched[e]];
    __syncthreads();
    const DeBlockDesc& d = s_desc;
    bool ok;
    if constexpr (CGK == 16)
      ok = de_block<TIER, 16, OBJ, MODEL, SK, false>(d, rank, a.k, ring, gg, sm, a, &s_abort, s_nrep);
    else if (TIER == TIER_F64 && d.cg == 16)
      ok = de_block<TIER, 16, OBJ, MODEL, SK>(d, rank, a.k, ring, gg, sm, a, &s_abort, s_nrep);
    else if (TIER == TIER_F64 && d.cg == 4)
      ok = de_block<TIER, 4, OBJ, MODEL, SK>(d, rank, a.k, ring, gg, sm, a, &s_abort, s_nrep);
    else ok = de_block<TIER, 8, OBJ, MODEL, SK>(d, rank, a.k, ring, gg, sm, a, &s_abort, s_nrep);
    if (!ok) return;
  }
}

}  // namespace pt
