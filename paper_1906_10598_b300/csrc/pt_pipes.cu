// Pipe-rate microbenchmarks of this GPU: the roofline denominators of the
// objective (no counterpart in the paper, which reports times only).
//
// The objective's sample loop issues one SFU cosine (__cosf) per
// sample-evaluation next to a few FP32 FMA-pipe instructions, and the DE's
// trial generation runs on the FP64 pipe. Each kernel here keeps one pipe
// busy with independent chains and measures, per SM, the operations retired
// per SM clock (clock64 between two CTA barriers, one CTA of 1024 threads per
// SM) and, for the whole GPU, operations per second (CUDA events):
//   PT_PIPE_COS   back-to-back __cosf, each with `nffma` extra FP32 FMAs
//                 (0: the cosine alone);
//   PT_PIPE_FFMA  FP32 FMAs alone (the FMA pipe and the issue rate);
//   PT_PIPE_DFMA  FP64 FMAs alone;
//   PT_PIPE_EX2   back-to-back ex2.approx (another SFU function).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pt_internal.h"

namespace {

constexpr int PIPE_THREADS = 1024;
constexpr int CHAINS = 8;  // independent chains per thread

// Keeps every value live without letting the compiler drop any operation.
__device__ __forceinline__ void sink(float v, float* out) {
  if (v == 12345.678f) out[threadIdx.x] = v;
}
__device__ __forceinline__ void sink_d(double v, float* out) {
  if (v == 12345.678) out[threadIdx.x] = (float)v;
}

// One CTA per SM (the dynamic shared memory the launch requests keeps a second
// CTA off), `iters` rounds of CHAINS cosines per thread, each followed by
// NF FP32 FMAs on separate accumulators.
template <int NF>
__global__ void __launch_bounds__(PIPE_THREADS, 1)
    k_pipe_cos(float x0, float a, float b, int iters, float* out, unsigned long long* cycles) {
  float x[CHAINS], y[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) {
    x[k] = x0 + 0.01f * (float)k + 1e-6f * (float)threadIdx.x;
    y[k] = 0.5f + 0.01f * (float)k;
  }
  __syncthreads();
  const unsigned long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) {
      x[k] = __cosf(x[k]);
#pragma unroll
      for (int f = 0; f < NF; ++f) y[(k + f) % CHAINS] = fmaf(y[(k + f) % CHAINS], a, b);
    }
  }
  __syncthreads();
  const unsigned long long c1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k] + y[k];
  sink(s, out);
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

// Back-to-back ex2.approx (another SFU function), for comparison with the cosine.
__global__ void __launch_bounds__(PIPE_THREADS, 1)
    k_pipe_ex2(float x0, float a, float b, int iters, float* out, unsigned long long* cycles) {
  float x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = x0 + 0.01f * (float)k + 1e-6f * (float)threadIdx.x;
  __syncthreads();
  const unsigned long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) {
      // 2^-x keeps the chain in (0.5, 1)
      const float nx = -x[k];
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(nx));
    }
  }
  __syncthreads();
  const unsigned long long c1 = clock64();
  float s = a + b;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  sink(s, out);
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

__global__ void __launch_bounds__(PIPE_THREADS, 1)
    k_pipe_ffma(float x0, float a, float b, int iters, float* out, unsigned long long* cycles) {
  float y[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) y[k] = x0 + 0.01f * (float)k + 1e-6f * (float)threadIdx.x;
  __syncthreads();
  const unsigned long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) y[k] = fmaf(y[k], a, b);
  }
  __syncthreads();
  const unsigned long long c1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += y[k];
  sink(s, out);
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

__global__ void __launch_bounds__(PIPE_THREADS, 1)
    k_pipe_dfma(double x0, double a, double b, int iters, float* out, unsigned long long* cycles) {
  double y[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) y[k] = x0 + 0.01 * (double)k + 1e-9 * (double)threadIdx.x;
  __syncthreads();
  const unsigned long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) y[k] = fma(y[k], a, b);
  }
  __syncthreads();
  const unsigned long long c1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += y[k];
  sink_d(s, out);
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

template <typename K>
cudaError_t launch_pipe(K kernel, int sms, size_t smem, int iters, float* out, unsigned long long* cyc) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<sms, PIPE_THREADS, smem>>>(0.3f, 0.999f, 1e-3f, iters, out, cyc);
  return cudaGetLastError();
}

}  // namespace

extern "C" int pt_pipe_rate(int device, int kind, int nffma, double* per_clk_sm, double* per_s, double* sm_mhz) {
  if (!per_clk_sm || !per_s || !sm_mhz) return PT_EINVAL;
  if (kind != PT_PIPE_COS && kind != PT_PIPE_FFMA && kind != PT_PIPE_DFMA && kind != PT_PIPE_EX2) return PT_EINVAL;
  if (kind == PT_PIPE_COS && nffma != 0 && nffma != 2 && nffma != 4 && nffma != 6 && nffma != 8) return PT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return PT_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return PT_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return PT_ECUDA;
  const int sms = prop.multiProcessorCount;
  // more than half of an SM's shared memory: one CTA per SM
  const size_t smem = std::min<size_t>(prop.sharedMemPerBlockOptin, prop.sharedMemPerMultiprocessor / 2 + 1024);
  // a few ms to ~20 ms per launch at the expected rates
  const int iters = kind == PT_PIPE_DFMA ? 1024 : kind == PT_PIPE_FFMA ? 65536 : 16384;
  float* d_out = nullptr;
  unsigned long long* d_cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PT_OK;
  std::vector<unsigned long long> cyc(sms);
  double best_s = 1e30, best_clk = 0.0, best_mhz = 0.0;
  if (cudaMalloc(&d_out, PIPE_THREADS * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&d_cyc, sms * sizeof(unsigned long long)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = PT_ECUDA;
  }
  // one untimed launch (module load, clocks ramping), then the best of five
  for (int rep = 0; rc == PT_OK && rep < 6; ++rep) {
    cudaError_t e = cudaEventRecord(e0);
    if (e == cudaSuccess) {
      if (kind == PT_PIPE_FFMA) e = launch_pipe(k_pipe_ffma, sms, smem, iters, d_out, d_cyc);
      else if (kind == PT_PIPE_EX2) e = launch_pipe(k_pipe_ex2, sms, smem, iters, d_out, d_cyc);
      else if (kind == PT_PIPE_DFMA) {
        e = cudaFuncSetAttribute(k_pipe_dfma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
          k_pipe_dfma<<<sms, PIPE_THREADS, smem>>>(0.3, 0.999, 1e-3, iters, d_out, d_cyc);
          e = cudaGetLastError();
        }
      } else if (nffma == 0) e = launch_pipe(k_pipe_cos<0>, sms, smem, iters, d_out, d_cyc);
      else if (nffma == 2) e = launch_pipe(k_pipe_cos<2>, sms, smem, iters, d_out, d_cyc);
      else if (nffma == 4) e = launch_pipe(k_pipe_cos<4>, sms, smem, iters, d_out, d_cyc);
      else if (nffma == 6) e = launch_pipe(k_pipe_cos<6>, sms, smem, iters, d_out, d_cyc);
      else e = launch_pipe(k_pipe_cos<8>, sms, smem, iters, d_out, d_cyc);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
      e = cudaMemcpy(cyc.data(), d_cyc, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rc = PT_ECUDA;
      break;
    }
    if (rep == 0) continue;
    std::vector<unsigned long long> sorted = cyc;
    std::sort(sorted.begin(), sorted.end());
    const double med_cyc = (double)sorted[sms / 2];
    const double ops_per_sm = (double)PIPE_THREADS * CHAINS * iters;
    const double sec = ms * 1e-3;
    if (sec < best_s) {
      best_s = sec;
      best_clk = ops_per_sm / med_cyc;
      best_mhz = med_cyc / sec * 1e-6;
    }
  }
  if (rc == PT_OK) {
    *per_clk_sm = best_clk;
    *per_s = (double)sms * PIPE_THREADS * CHAINS * iters / best_s;
    *sm_mhz = best_mhz;
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_out) cudaFree(d_out);
  if (d_cyc) cudaFree(d_cyc);
  return rc;
}
