// Kernels of the phase-tracking hot path (arxiv 1906.10598, Sec. 1.2-2.2):
//   k_absmax      max |stored sample| of a loaded block (sets the SSE fixed-point scale)
//   k_objective   Eq. 2-2-4 for a fixed candidate set (tiles x candidate batches)
//   k_finalize    fixed-point accumulators -> FP64 SSE
//   k_de          persistent DE/rand/1/bin solve of one block (Table 3-1-1 controls)
//
// Work decomposition shared by the objective and DE kernels: a CTA owns a
// contiguous range of 256-sample tiles, staged once into shared memory by a
// bulk (TMA) copy and converted to the compute type; a work item is one tile
// x 8 candidates, run by one warp with 8 consecutive samples per lane in
// registers. Per-item FP32 sums are reduced across the warp and added, as
// 64-bit fixed point with a per-candidate scale, to shared and then global
// accumulators. Integer addition is exact and associative, so the SSE does not
// depend on the launch shape, the CTA count or the order of completion.
#pragma once

#include "pt_device.cuh"

namespace pt {

constexpr int NT = 512;        // threads per CTA of the objective / DE kernels
constexpr int CAND_BYTES = 64; // per-candidate prepared data in shared memory

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
template <int TIER>
__device__ __forceinline__ void prep_candidate(const double* th, const BlockArgs& b, unsigned char* cdata,
                                               float* negA, int* kexp) {
  *negA = -__double2float_rn(th[0]);
  *kexp = sse_scale_exp(b.n, b.smax, th[0]);
  if (TIER == TIER_F64) {
    Poly P = make_poly(th, b);
    u128* e = reinterpret_cast<u128*>(cdata);
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = P.e[k];
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

__device__ __forceinline__ void prep_zero(unsigned char* cdata, float* negA, int* kexp) {
  *negA = 0.f;
  *kexp = 0;
  uint4* p = reinterpret_cast<uint4*>(cdata);
#pragma unroll
  for (int k = 0; k < CAND_BYTES / 16; ++k) p[k] = make_uint4(0, 0, 0, 0);
}

// ---------------------------------------------------------------------------
// Work items.

// Default tier: 32-bit fixed-point phase walk + FP32 small terms + SFU cosine.
template <bool MASKED>
__device__ __forceinline__ void item_f64(const float (&s)[M], const uint4* anc_t, const float* negA, int g, int lane,
                                         int nvalid, const float (&kk)[M], const float (&kkk)[M], float (&acc)[CG]) {
#pragma unroll
  for (int c = 0; c < CG; ++c) {
    const int cand = g * CG + c;
    const uint4 a = anc_t[cand];
    const float nA = negA[cand];
    const uint32_t V = a.y;
    uint32_t u = a.x + (uint32_t)(lane * M) * V;
    const float E2 = __uint_as_float(a.z), E3 = __uint_as_float(a.w);
    float sum = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const float q = fmaf(kkk[m], E3, kk[m] * E2);
      const float x = fmaf((float)(int)u, TWO_PI_2M32, q);
      const float cv = __cosf(x);
      float r = fmaf(nA, cv, s[m]);
      if (MASKED) r = (lane * M + m < nvalid) ? r : 0.f;
      sum = fmaf(r, r, sum);
      u += V;
    }
    acc[c] = sum;
  }
}

// All-FP64 tier: Horner phase in seconds, reduction mod 1, FP64 cospi.
template <bool MASKED>
__device__ __forceinline__ void item_plain(const double (&s)[M], const unsigned char* cdata, int g, int lane,
                                           int nvalid, int64_t tstart, const BlockArgs& b, double (&acc)[CG]) {
#pragma unroll 1
  for (int c = 0; c < CG; ++c) {
    const double* k = reinterpret_cast<const double*>(cdata + (g * CG + c) * CAND_BYTES);
    const double A = k[0], c0 = k[1], c1 = k[2], c2 = k[3], c3 = k[4];
    double sum = 0.0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int64_t i = tstart + lane * M + m;
      const double t = fma((double)i, b.h, b.t0);
      const double p = fma(fma(fma(c3, t, c2), t, c1), t, c0);
      const double r = p - rint(p);
      const double cv = cospi(2.0 * r);
      double res = fma(-A, cv, s[m]);
      if (MASKED) res = (lane * M + m < nvalid) ? res : 0.0;
      sum = fma(res, res, sum);
    }
    acc[c] = sum;
  }
}

// Double-float tier: per-sample phase in double-float, FP32 cosine.
template <bool MASKED>
__device__ __forceinline__ void item_df32(const float (&s)[M], const unsigned char* cdata, const float* negA, int g,
                                          int lane, int nvalid, int64_t tstart, dfloat t0d, dfloat hd,
                                          float (&acc)[CG]) {
#pragma unroll 1
  for (int c = 0; c < CG; ++c) {
    const dfloat* k = reinterpret_cast<const dfloat*>(cdata + (g * CG + c) * CAND_BYTES);
    const dfloat c0 = k[0], c1 = k[1], c2 = k[2], c3 = k[3];
    const float nA = negA[g * CG + c];
    float sum = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int64_t i = tstart + lane * M + m;
      // t = t0 + i h in double-float (i < 2^24 is exact in FP32)
      const dfloat t = df_add(t0d, df_mul({(float)i, 0.f}, hd));
      dfloat p = df_add(df_mul(c3, t), c2);
      p = df_add(df_mul(p, t), c1);
      p = df_add(df_mul(p, t), c0);
      const float rh = p.hi - rintf(p.hi);
      const float r = rh + p.lo;
      const float cv = __cosf(r * 6.28318530717958648f);
      float res = fmaf(nA, cv, s[m]);
      if (MASKED) res = (lane * M + m < nvalid) ? res : 0.f;
      sum = fmaf(res, res, sum);
    }
    acc[c] = sum;
  }
}

// Naive FP32 tier: Horner phase in seconds in FP32.
template <bool MASKED>
__device__ __forceinline__ void item_f32(const float (&s)[M], const unsigned char* cdata, const float* negA, int g,
                                         int lane, int nvalid, int64_t tstart, float t0f, float hf,
                                         float (&acc)[CG]) {
#pragma unroll 1
  for (int c = 0; c < CG; ++c) {
    const float* k = reinterpret_cast<const float*>(cdata + (g * CG + c) * CAND_BYTES);
    const float c0 = k[0], c1 = k[1], c2 = k[2], c3 = k[3];
    const float nA = negA[g * CG + c];
    float sum = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int64_t i = tstart + lane * M + m;
      const float t = fmaf((float)i, hf, t0f);
      const float p = fmaf(fmaf(fmaf(c3, t, c2), t, c1), t, c0);
      const float r = p - rintf(p);
      const float cv = __cosf(r * 6.28318530717958648f);
      float res = fmaf(nA, cv, s[m]);
      if (MASKED) res = (lane * M + m < nvalid) ? res : 0.f;
      sum = fmaf(res, res, sum);
    }
    acc[c] = sum;
  }
}

// Evaluate candidates [0, ncand) (prepared in cdata/negA/kexp, padded to npad,
// a multiple of CG) on the CTA's tiles [tile_begin, tile_begin + ntiles_cta)
// whose converted samples are s32 / s64 (indexed from tile_begin). Adds the
// fixed-point partial SSE of each candidate into acc[cand] (shared).
// anc: shared scratch for tiles_chunk x npad anchors. Ends with __syncthreads().
template <int TIER>
__device__ void eval_range(const BlockArgs& b, int64_t tile_begin, int ntiles_cta, const float* s32,
                           const double* s64, const unsigned char* cdata, const float* negA, const int* kexp,
                           int ncand, int npad, uint4* anc, int tiles_chunk, unsigned long long* acc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int G = npad / CG;
  float kk[M], kkk[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int k = lane * M + m;
    kk[m] = (float)(k * k);
    kkk[m] = (float)(k * k * k);
  }
  const dfloat t0d = df_from_double(b.t0), hd = df_from_double(b.h);
  const float t0f = __double2float_rn(b.t0), hf = __double2float_rn(b.h);

  for (int cbeg = 0; cbeg < ntiles_cta; cbeg += tiles_chunk) {
    const int nt = min(tiles_chunk, ntiles_cta - cbeg);
    if (TIER == TIER_F64) {
      for (int idx = tid; idx < nt * npad; idx += blockDim.x) {
        const int t = idx / npad, c = idx - t * npad;
        uint4 a = make_uint4(0, 0, 0, 0);
        if (c < ncand) {
          const u128* e = reinterpret_cast<const u128*>(cdata + c * CAND_BYTES);
          Poly P;
          P.e[0] = e[0];
          P.e[1] = e[1];
          P.e[2] = e[2];
          P.e[3] = e[3];
          a = make_anchor(P, (uint64_t)(tile_begin + cbeg + t) * (uint64_t)L);
        }
        anc[idx] = a;
      }
      __syncthreads();
    }
    for (int it = warp; it < nt * G; it += nw) {
      const int t = it / G, g = it - t * G;
      const int64_t tstart = (tile_begin + cbeg + t) * (int64_t)L;
      const int64_t rem = b.n - tstart;
      const int nvalid = rem < L ? (int)rem : L;
      const int64_t soff = (int64_t)(cbeg + t) * L + lane * M;
      int cand = g * CG + (lane >> 2);
      if (TIER == TIER_PLAIN) {
        double s[M];
#pragma unroll
        for (int m = 0; m < M; m += 2) {
          const double2 v = *reinterpret_cast<const double2*>(s64 + soff + m);
          s[m] = v.x;
          s[m + 1] = v.y;
        }
        double acc8[CG];
        if (nvalid == L) item_plain<false>(s, cdata, g, lane, nvalid, tstart, b, acc8);
        else item_plain<true>(s, cdata, g, lane, nvalid, tstart, b, acc8);
        const double z = warp_reduce_scatter8(acc8, lane);
        if ((lane & 3) == 0 && cand < ncand) {
          const long long v = __double2ll_rn(ldexp(z, kexp[cand]));
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
        float acc8[CG];
        if (TIER == TIER_F64) {
          const uint4* anc_t = anc + t * npad;
          if (nvalid == L) item_f64<false>(s, anc_t, negA, g, lane, nvalid, kk, kkk, acc8);
          else item_f64<true>(s, anc_t, negA, g, lane, nvalid, kk, kkk, acc8);
        } else if (TIER == TIER_DF32) {
          if (nvalid == L) item_df32<false>(s, cdata, negA, g, lane, nvalid, tstart, t0d, hd, acc8);
          else item_df32<true>(s, cdata, negA, g, lane, nvalid, tstart, t0d, hd, acc8);
        } else {
          if (nvalid == L) item_f32<false>(s, cdata, negA, g, lane, nvalid, tstart, t0f, hf, acc8);
          else item_f32<true>(s, cdata, negA, g, lane, nvalid, tstart, t0f, hf, acc8);
        }
        const float z = warp_reduce_scatter8(acc8, lane);
        if ((lane & 3) == 0 && cand < ncand) {
          const long long v = __float2ll_rn(z * exp2_int_f(kexp[cand]));
          atomicAdd(&acc[cand], (unsigned long long)v);
        }
      }
    }
    __syncthreads();
  }
}

// Stage tiles [tb, tb + nt) of the block into shared memory and convert them.
// Returns false (and sets *err) if the bulk copy did not complete in time.
template <int TIER>
__device__ bool stage_tiles(const BlockArgs& b, int64_t tb, int nt, void* raw, float* s32, double* s64,
                            uint64_t* mbar, uint64_t timeout_ns, int* err) {
  const uint32_t bytes = (uint32_t)nt * (uint32_t)L * (uint32_t)b.esize;
  const char* src = reinterpret_cast<const char*>(b.samples) + tb * (int64_t)L * b.esize;
  if (!bulk_stage(raw, src, bytes, mbar, timeout_ns)) {
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
  size_t off_mbar, off_cdata, off_negA, off_kexp, off_acc, off_anc, off_samp, off_raw, off_pop, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// npad: padded candidates; tmax: max tiles per CTA; chunk: anchor tile chunk;
// pop: population slots (0 for the objective kernel).
__host__ __device__ inline SmemLayout smem_layout(int tier, int npad, int tmax, int chunk, int esize, int pop) {
  SmemLayout s;
  size_t o = 0;
  s.off_mbar = o;
  o += 16;
  s.off_pop = o;
  o += align_up((size_t)pop * (2 * D + 1) * sizeof(double), 16);
  s.off_cdata = o;
  o += (size_t)npad * CAND_BYTES;
  s.off_negA = o;
  o += align_up((size_t)npad * sizeof(float), 16);
  s.off_kexp = o;
  o += align_up((size_t)npad * sizeof(int), 16);
  s.off_acc = o;
  o += align_up((size_t)npad * sizeof(unsigned long long), 16);
  s.off_anc = o;
  o += (tier == TIER_F64) ? (size_t)chunk * npad * sizeof(uint4) : 0;
  s.off_samp = o;
  o += align_up((size_t)tmax * L * (tier_uses_f64_samples(tier) ? 8 : 4), 128);
  s.off_raw = o;
  o += align_up((size_t)tmax * L * esize, 128);
  s.total = o;
  return s;
}

// ---------------------------------------------------------------------------

__global__ void k_absmax(const void* samples, int64_t n, int dtype, unsigned long long* out) {
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
  int cpc;          // candidates per CTA, multiple of CG (grid.y)
  int tiles_chunk;
  unsigned long long* acc;  // [ncand], zeroed by the caller
  int* err;
  uint64_t timeout_ns;
};

template <int TIER>
__global__ void __launch_bounds__(NT, 1) k_objective(ObjArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t tb = (int64_t)blockIdx.x * a.tpc;
  const int nt = (int)min((int64_t)a.tpc, a.b.ntiles - tb);
  const int cb = blockIdx.y * a.cpc;
  const int nc = min(a.cpc, a.ncand - cb);
  if (nt <= 0 || nc <= 0) return;
  const int npad = (nc + CG - 1) / CG * CG;
  const SmemLayout S = smem_layout(TIER, npad, a.tpc, a.tiles_chunk, a.b.esize, 0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S.off_mbar);
  unsigned char* cdata = smem + S.off_cdata;
  float* negA = reinterpret_cast<float*>(smem + S.off_negA);
  int* kexp = reinterpret_cast<int*>(smem + S.off_kexp);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem + S.off_acc);
  uint4* anc = reinterpret_cast<uint4*>(smem + S.off_anc);
  float* s32 = reinterpret_cast<float*>(smem + S.off_samp);
  double* s64 = reinterpret_cast<double*>(smem + S.off_samp);
  void* raw = smem + S.off_raw;

  const int tid = threadIdx.x;
  if (tid < npad) {
    acc[tid] = 0ull;
    if (tid < nc) {
      double th[D];
#pragma unroll
      for (int j = 0; j < D; ++j) th[j] = a.cands[(int64_t)(cb + tid) * D + j];
      prep_candidate<TIER>(th, a.b, cdata + tid * CAND_BYTES, negA + tid, kexp + tid);
    } else {
      prep_zero(cdata + tid * CAND_BYTES, negA + tid, kexp + tid);
    }
  }
  if (!stage_tiles<TIER>(a.b, tb, nt, raw, s32, s64, mbar, a.timeout_ns, a.err)) return;
  eval_range<TIER>(a.b, tb, nt, s32, s64, cdata, negA, kexp, nc, npad, anc, a.tiles_chunk, acc);
  if (tid < nc) atomicAdd(&a.acc[cb + tid], acc[tid]);
}

__global__ void k_finalize(const double* cands, int ncand, const unsigned long long* acc, int64_t n, double smax,
                           double* sse) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand) return;
  const int k = sse_scale_exp(n, smax, cands[(int64_t)c * D]);
  sse[c] = ldexp((double)(long long)acc[c], -k);
}

struct DeArgs {
  BlockArgs b;
  DeControls dc;
  int np, npad, gens;
  int nctas;
  int tmax;
  int tiles_chunk;
  unsigned long long* gacc;  // [3][npad], zeroed by the caller
  unsigned* bar;             // arrival counter, zeroed by the caller
  int* err;                  // zeroed by the caller
  double* out;               // [6]
  double* pop_out;           // [np * 5] (device)
  double* fit_out;           // [np] (device)
  uint64_t timeout_ns;
};

// Persistent DE solve: every CTA holds the whole population and generates
// every trial itself (identical Philox draws, identical FP64 arithmetic), so
// the only exchange is the per-generation fixed-point SSE sums, added with
// global atomics into a 3-deep ring and read back after one grid barrier.
// Launched cooperatively (all CTAs co-resident); every wait is bounded.
template <int TIER>
__global__ void __launch_bounds__(NT, 1) k_de(DeArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout S = smem_layout(TIER, a.npad, a.tmax, a.tiles_chunk, a.b.esize, a.npad);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S.off_mbar);
  double* x = reinterpret_cast<double*>(smem + S.off_pop);
  double* u = x + a.npad * D;
  double* fx = u + a.npad * D;
  unsigned char* cdata = smem + S.off_cdata;
  float* negA = reinterpret_cast<float*>(smem + S.off_negA);
  int* kexp = reinterpret_cast<int*>(smem + S.off_kexp);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem + S.off_acc);
  uint4* anc = reinterpret_cast<uint4*>(smem + S.off_anc);
  float* s32 = reinterpret_cast<float*>(smem + S.off_samp);
  double* s64 = reinterpret_cast<double*>(smem + S.off_samp);
  void* raw = smem + S.off_raw;
  __shared__ int s_abort;

  const int tid = threadIdx.x, bid = blockIdx.x;
  const int64_t tb = (int64_t)bid * a.b.ntiles / a.nctas;
  const int nt = (int)((int64_t)(bid + 1) * a.b.ntiles / a.nctas - tb);
  if (!stage_tiles<TIER>(a.b, tb, nt, raw, s32, s64, mbar, a.timeout_ns, a.err)) return;

  for (int gen = 0; gen <= a.gens; ++gen) {
    const int ring = gen % 3;
    if (tid < a.npad) {
      acc[tid] = 0ull;
      if (tid < a.np) {
        double* ui = u + tid * D;
        if (gen == 0) de_init(a.dc, tid, ui);
        else de_trial(a.dc, x, a.np, tid, (uint32_t)gen, ui);
        prep_candidate<TIER>(ui, a.b, cdata + tid * CAND_BYTES, negA + tid, kexp + tid);
      } else {
        prep_zero(cdata + tid * CAND_BYTES, negA + tid, kexp + tid);
      }
    }
    __syncthreads();
    eval_range<TIER>(a.b, tb, nt, s32, s64, cdata, negA, kexp, a.np, a.npad, anc, a.tiles_chunk, acc);
    if (tid < a.np) {
      atomicAdd(&a.gacc[ring * a.npad + tid], acc[tid]);
      // the slot of generation gen+1 was last read before barrier gen-1: clear it
      if (bid == 0) a.gacc[((gen + 1) % 3) * a.npad + tid] = 0ull;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(a.bar, 1u);
      const unsigned target = (unsigned)(gen + 1) * (unsigned)a.nctas;
      const uint64_t t_start = globaltimer_ns();
      int abort = 0;
      while (ld_acquire_u32(a.bar) < target) {
        if (ld_volatile_i32(a.err) != DEV_OK) {
          abort = 1;
          break;
        }
        if (globaltimer_ns() - t_start > a.timeout_ns) {
          atomicExch(a.err, DEV_TIMEOUT);
          abort = 1;
          break;
        }
      }
      s_abort = abort;
    }
    __syncthreads();
    if (s_abort) return;
    if (tid < a.np) {
      const unsigned long long v = __ldcg(&a.gacc[ring * a.npad + tid]);
      const double f = ldexp((double)(long long)v, -kexp[tid]);
      if (gen == 0 || f <= fx[tid]) {
        fx[tid] = f;
#pragma unroll
        for (int j = 0; j < D; ++j) x[tid * D + j] = u[tid * D + j];
      }
    }
    __syncthreads();
  }
  if (bid == 0) {
    if (tid == 0) {
      int best = 0;
      for (int i = 1; i < a.np; ++i)
        if (fx[i] < fx[best]) best = i;
      for (int j = 0; j < D; ++j) a.out[j] = x[best * D + j];
      a.out[D] = fx[best];
    }
    for (int i = tid; i < a.np * D; i += blockDim.x) a.pop_out[i] = x[i];
    for (int i = tid; i < a.np; i += blockDim.x) a.fit_out[i] = fx[i];
  }
}

}  // namespace pt
