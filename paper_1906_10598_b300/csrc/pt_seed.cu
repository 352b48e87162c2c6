// FFT seed of the first block's ranges (Sec. 3.1.1): the frequency at the
// block centre from the spectrum of a small piece of data there, its rate by
// a central difference of three such frequencies, the amplitude from the
// spectral peak; ranges f0 and A +- f0_rel, c3 in [-50, 50] rad/s^3, c5 +-
// 0.2 c4 / T.
//
// k_seed_pieces: one CTA per piece (three pieces of Np samples starting at
// n/2 - Np/2 + (k - 1) Np): periodic Hann window, radix-2 FFT in shared
// memory (FP32 complex, Np <= 8192), argmax of |X|^2 over bins 1 .. Np/2 - 1
// (lowest index on ties), and the peak's offset from a parabola through the
// log magnitudes of the peak bin and its neighbours (FP64).
// k_seed_finish: the estimates and the ranges from the three peaks.
#include <cuda_runtime.h>

#include <cmath>

#include "pt_device.cuh"
#include "pt_internal.h"

namespace pt {
namespace {

constexpr int SEED_NT = 512;
constexpr int SEED_NP_MAX = 8192;

struct SeedPeak {
  int bin;
  double delta;   // refined offset from bin (bins)
  double power;   // |X[bin]|^2
};

__device__ __forceinline__ unsigned bit_reverse(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

__global__ void __launch_bounds__(SEED_NT) k_seed_pieces(const void* samples, int64_t n, int dtype, double scale,
                                                         int np, int log2np, SeedPeak* out) {
  extern __shared__ float2 buf[];
  __shared__ float s_p[SEED_NT / 32];
  __shared__ int s_k[SEED_NT / 32];
  const int tid = threadIdx.x;
  const int64_t start = n / 2 - np / 2 + ((int64_t)blockIdx.x - 1) * np;
  // windowed samples in bit-reversed order
  for (int j = tid; j < np; j += blockDim.x) {
    const float w = 0.5f - 0.5f * cospif(2.0f * (float)j / (float)np);
    const float v = (float)load_physical(samples, dtype, start + j, scale);
    buf[bit_reverse((unsigned)j, log2np)] = make_float2(w * v, 0.f);
  }
  __syncthreads();
  // decimation-in-time butterflies, X_k = sum_j x_j exp(-2 pi i j k / np)
  for (int half = 1; half < np; half <<= 1) {
    const int len = half << 1;
    for (int b = tid; b < np / 2; b += blockDim.x) {
      const int q = b & (half - 1);
      const int i = (b / half) * len + q;
      float sn, cs;
      sincospif(-(float)q / (float)half, &sn, &cs);
      const float2 u = buf[i], x = buf[i + half];
      const float2 v = make_float2(x.x * cs - x.y * sn, x.x * sn + x.y * cs);
      buf[i] = make_float2(u.x + v.x, u.y + v.y);
      buf[i + half] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
  // argmax of the power over bins 1 .. np/2 - 1 (lowest index on ties)
  float best = -1.f;
  int bk = 0;
  for (int k = 1 + tid; k < np / 2; k += blockDim.x) {
    const float2 z = buf[k];
    const float p = z.x * z.x + z.y * z.y;
    if (p > best) {
      best = p;
      bk = k;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float p2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int k2 = __shfl_xor_sync(0xffffffffu, bk, o);
    if (p2 > best || (p2 == best && k2 < bk)) {
      best = p2;
      bk = k2;
    }
  }
  if ((tid & 31) == 0) {
    s_p[tid >> 5] = best;
    s_k[tid >> 5] = bk;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (s_p[w] > best || (s_p[w] == best && s_k[w] < bk)) {
        best = s_p[w];
        bk = s_k[w];
      }
    auto power = [&](int k) {
      const float2 z = buf[k];
      return (double)z.x * z.x + (double)z.y * z.y;
    };
    // parabola through ln|X| at bk - 1, bk, bk + 1 (ln|X| = ln(P) / 2; the factor cancels)
    const double a = log(power(bk - 1)), b = log(power(bk)), g = log(power(bk + 1));
    const double den = a - 2.0 * b + g;
    SeedPeak r;
    r.bin = bk;
    r.delta = den < 0.0 ? 0.5 * (a - g) / den : 0.0;
    r.power = power(bk);
    out[blockIdx.x] = r;
  }
}

// The estimates and the ranges (pt_seed_result) from the three refined peaks.
__global__ void k_seed_finish(const SeedPeak* pk, int64_t n, double fs, double t0, int np, double f0_rel,
                              pt_seed_result* out) {
  pt_seed_result r{};
  r.piece_len = np;
  for (int k = 0; k < 3; ++k) {
    const int64_t start = n / 2 - np / 2 + (int64_t)(k - 1) * np;
    r.peak_bin[k] = pk[k].bin;
    r.peak_delta[k] = pk[k].delta;
    r.piece_freq[k] = ((double)pk[k].bin + pk[k].delta) * fs / (double)np;
    r.piece_time[k] = t0 + (double)(start + np / 2) / fs;
  }
  r.f1 = (r.piece_freq[2] - r.piece_freq[0]) / (r.piece_time[2] - r.piece_time[0]);
  r.f0 = r.piece_freq[1] - r.f1 * r.piece_time[1];
  // the periodic Hann window sums to np/2; its response at offset d is sinc(d) / (1 - d^2)
  const double d = pk[1].delta;
  const double resp = (d == 0.0 ? 1.0 : sinpi(d) / (3.14159265358979323846 * d)) / (1.0 - d * d);
  r.A = 2.0 * sqrt(pk[1].power) / (0.5 * (double)np * resp);
  const double T = (double)n / fs;
  const double f2_max = 3.0 * 50.0 / 3.14159265358979323846;  // c3 = pi f2 / 3 in [-50, 50] rad/s^3
  const double hw1 = fmax(f0_rel * fabs(r.f1), fs * fs / ((double)np * (double)np));
  const double b[14] = {(1.0 - f0_rel) * r.A, (1.0 + f0_rel) * r.A,
                        -3.14159265358979323846, 3.14159265358979323846,
                        r.f0 - f0_rel * fabs(r.f0), r.f0 + f0_rel * fabs(r.f0),
                        r.f1 - hw1, r.f1 + hw1,
                        -f2_max, f2_max,
                        -0.2 * r.A / T, 0.2 * r.A / T,
                        -192.0 / (T * T * T * T), 192.0 / (T * T * T * T)};
  for (int j = 0; j < 14; ++j) r.bounds[j] = b[j];
  *out = r;
}

}  // namespace
}  // namespace pt

using namespace pt;

extern "C" {

int pt_seed_bounds(pt_ctx* c, double f0_rel, int piece_len, pt_seed_result* out) {
  if (!c) return PT_EINVAL;
  if (!out || !(f0_rel > 0.0) || !(f0_rel < 1.0) || piece_len < 0)
    return fail(c, PT_EINVAL, "pt_seed_bounds: invalid argument");
  if (!c->has_block) return fail(c, PT_ENOBLOCK, "pt_seed_bounds: no block loaded");
  const int64_t n = c->blk.n;
  int np = piece_len;
  if (np == 0) {
    if (n < 64) return fail(c, PT_EINVAL, "pt_seed_bounds: block too short for three pieces");
    np = 1;
    while ((int64_t)np * 2 <= n / 4 && np * 2 <= SEED_NP_MAX) np *= 2;
  }
  int log2np = 0;
  while ((1 << log2np) < np) ++log2np;
  if (np < 16 || np > SEED_NP_MAX || (1 << log2np) != np || n / 2 - 3 * (int64_t)np / 2 < 0 ||
      n / 2 + 3 * (int64_t)np / 2 > n)
    return fail(c, PT_EINVAL, "pt_seed_bounds: block too short for three pieces");
  PT_CUDA(c, cudaSetDevice(c->device));
  if (!c->d_seed) PT_CUDA(c, cudaMalloc(&c->d_seed, 4096));
  SeedPeak* d_pk = reinterpret_cast<SeedPeak*>(c->d_seed);
  pt_seed_result* d_res = reinterpret_cast<pt_seed_result*>(reinterpret_cast<char*>(c->d_seed) + 256);
  static_assert(3 * sizeof(SeedPeak) <= 256 && 256 + sizeof(pt_seed_result) <= 4096, "seed scratch layout");
  const size_t smem = (size_t)np * sizeof(float2);
  PT_CUDA(c, cudaFuncSetAttribute(k_seed_pieces, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_seed_pieces<<<3, SEED_NT, smem, c->stream>>>(c->blk.samples, n, c->blk.dtype, c->blk.scale, np, log2np, d_pk);
  PT_CUDA(c, cudaGetLastError());
  k_seed_finish<<<1, 1, 0, c->stream>>>(d_pk, n, c->blk.fs, c->blk.t0, np, f0_rel, d_res);
  PT_CUDA(c, cudaGetLastError());
  PT_CUDA(c, cudaMemcpyAsync(out, d_res, sizeof(pt_seed_result), cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(c, cudaStreamSynchronize(c->stream));
  return PT_OK;
}

}  // extern "C"
