// C ABI of the phase-tracking hot path (declarations and contracts in
// include/phasetrack.h). Host side: argument validation, device buffers,
// launch shapes and the synchronous call protocol. Every step of the
// computation runs in the kernels of pt_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/phasetrack.h"
#include "pt_kernels.cuh"

using namespace pt;

struct pt_ctx {
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  // loaded block
  void* d_samples = nullptr;
  size_t samples_cap = 0;
  BlockArgs blk{};
  bool has_block = false;
  // objective scratch
  unsigned long long* d_acc = nullptr;
  size_t acc_cap = 0;
  double* d_cands = nullptr;
  size_t cands_cap = 0;
  double* d_sse = nullptr;
  size_t sse_cap = 0;
  // DE scratch (sized for PT_POP_MAX)
  unsigned long long* d_gacc = nullptr;
  unsigned* d_bar = nullptr;
  int* d_err = nullptr;
  double* d_out = nullptr;
  double* d_pop = nullptr;
  double* d_fit = nullptr;
  unsigned long long* d_u64 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.f;
  uint64_t timeout_ns = 2000000000ull;
};

namespace {

int fail(pt_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define PT_CUDA(ctx, call)                                                                      \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    }                                                                                           \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int esize_of(int dtype) {
  switch (dtype) {
    case PT_I8: return 1;
    case PT_I16: return 2;
    case PT_F16: return 2;
    case PT_F32: return 4;
    case PT_F64: return 8;
    default: return 0;
  }
}

template <typename T>
int ensure(pt_ctx* c, T** p, size_t* cap, size_t count) {
  if (*cap >= count) return PT_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  PT_CUDA(c, cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)));
  *cap = count;
  return PT_OK;
}

bool valid_tier(int t) { return t >= PT_TIER_F64 && t <= PT_TIER_F32; }

int kernel_error(pt_ctx* c) {
  int h_err = 0;
  PT_CUDA(c, cudaMemcpyAsync(&h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h_err == DEV_TIMEOUT) return fail(c, PT_ETIMEOUT, "a bounded device-side wait expired");
  if (h_err != DEV_OK) return fail(c, PT_ECUDA, "device error status " + std::to_string(h_err));
  return PT_OK;
}

// Candidates per work item for the default tier: the width in {16, 8, 4}
// that pads `n` the least (wider on ties); the other tiers use 8.
int pick_cg(int tier, int n) {
  if (tier != PT_TIER_F64) return 8;
  int best = 16, best_pad = (n + 15) / 16 * 16;
  for (int cg : {8, 4}) {
    const int pad = (n + cg - 1) / cg * cg;
    if (pad < best_pad) {
      best = cg;
      best_pad = pad;
    }
  }
  return best;
}

// ---- objective -------------------------------------------------------------

template <int TIER, int CGV>
int launch_objective(pt_ctx* c, const double* d_cands, int ncand) {
  const BlockArgs& b = c->blk;
  ObjArgs a{};
  a.b = b;
  a.cands = d_cands;
  a.ncand = ncand;
  a.cpc = std::min(((ncand + CGV - 1) / CGV) * CGV, NP_MAX);
  const int ny = (ncand + a.cpc - 1) / a.cpc;
  // about two CTAs per SM in total, tiles split evenly
  const int64_t want = 2LL * c->sms;
  int64_t tpc = (b.ntiles * ny + want - 1) / want;
  tpc = std::max<int64_t>(1, std::min<int64_t>(tpc, 32));
  a.tpc = (int)tpc;
  const int nx = (int)((b.ntiles + a.tpc - 1) / a.tpc);
  a.acc = c->d_acc;
  a.err = c->d_err;
  a.timeout_ns = c->timeout_ns;
  const SmemLayout S = smem_layout(TIER, a.cpc, a.tpc, CGV, b.esize, 0, NT);
  if (S.total > c->smem_optin) return fail(c, PT_EINVAL, "objective launch needs too much shared memory");
  PT_CUDA(c, cudaFuncSetAttribute(k_objective<TIER, CGV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)S.total));
  dim3 grid(nx, ny);
  k_objective<TIER, CGV><<<grid, NT, S.total, c->stream>>>(a);
  PT_CUDA(c, cudaGetLastError());
  return PT_OK;
}

int launch_objective_any(pt_ctx* c, int tier, const double* d_cands, int ncand) {
  switch (tier) {
    case PT_TIER_F64: {
      const int cg = pick_cg(tier, std::min(ncand, NP_MAX));
      if (cg == 16) return launch_objective<TIER_F64, 16>(c, d_cands, ncand);
      if (cg == 8) return launch_objective<TIER_F64, 8>(c, d_cands, ncand);
      return launch_objective<TIER_F64, 4>(c, d_cands, ncand);
    }
    case PT_TIER_PLAIN: return launch_objective<TIER_PLAIN, 8>(c, d_cands, ncand);
    case PT_TIER_DF32: return launch_objective<TIER_DF32, 8>(c, d_cands, ncand);
    default: return launch_objective<TIER_F32, 8>(c, d_cands, ncand);
  }
}

// ---- DE --------------------------------------------------------------------

template <int TIER, int CGV>
int launch_de(pt_ctx* c, DeArgs& a) {
  const BlockArgs& b = c->blk;
  a.npad = (a.np + CGV - 1) / CGV * CGV;
  a.nctas = (int)std::min<int64_t>(b.ntiles, c->sms);
  a.tmax = (int)((b.ntiles + a.nctas - 1) / a.nctas);
  const SmemLayout S = smem_layout(TIER, a.npad, a.tmax, CGV, b.esize, a.npad, NT);
  if (S.total > c->smem_optin)
    return fail(c, PT_EINVAL, "block too long for the resident DE kernel (" + std::to_string(S.total) +
                                  " bytes of shared memory per CTA)");
  PT_CUDA(c, cudaFuncSetAttribute(k_de<TIER, CGV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total));
  int occ = 0;
  PT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_de<TIER, CGV>, NT, S.total));
  if (occ < 1 || a.nctas > occ * c->sms) return fail(c, PT_EINVAL, "DE grid cannot be co-resident");
  void* args[] = {&a};
  PT_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_de<TIER, CGV>, dim3(a.nctas), dim3(NT), args, S.total,
                                         c->stream));
  return PT_OK;
}

int launch_de_any(pt_ctx* c, int tier, DeArgs& a) {
  switch (tier) {
    case PT_TIER_F64: {
      const int cg = pick_cg(tier, a.np);
      if (cg == 16) return launch_de<TIER_F64, 16>(c, a);
      if (cg == 8) return launch_de<TIER_F64, 8>(c, a);
      return launch_de<TIER_F64, 4>(c, a);
    }
    case PT_TIER_PLAIN: return launch_de<TIER_PLAIN, 8>(c, a);
    case PT_TIER_DF32: return launch_de<TIER_DF32, 8>(c, a);
    default: return launch_de<TIER_F32, 8>(c, a);
  }
}

}  // namespace

// ---- C ABI -------------------------------------------------------------------

extern "C" {

int pt_create(pt_ctx** out, int device) {
  if (!out) return PT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return PT_EINVAL;
  }
  pt_ctx* c = new (std::nothrow) pt_ctx();
  if (!c) return PT_ENOMEM;
  c->device = device;
  auto bad = [&](cudaError_t e) {
    if (e == cudaSuccess) return false;
    pt_destroy(c);
    return true;
  };
  if (bad(cudaSetDevice(device))) return PT_ECUDA;
  cudaDeviceProp prop;
  if (bad(cudaGetDeviceProperties(&prop, device))) return PT_ECUDA;
  c->sms = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  if (bad(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking))) return PT_ECUDA;
  c->stream = c->own_stream;
  if (bad(cudaMalloc(&c->d_gacc, 3 * PT_POP_MAX * sizeof(unsigned long long)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_bar, sizeof(unsigned)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_err, sizeof(int)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_out, 8 * sizeof(double)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_pop, PT_POP_MAX * D * sizeof(double)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_fit, PT_POP_MAX * sizeof(double)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_u64, sizeof(unsigned long long)))) return PT_ENOMEM;
  if (bad(cudaEventCreate(&c->ev0))) return PT_ECUDA;
  if (bad(cudaEventCreate(&c->ev1))) return PT_ECUDA;
  *out = c;
  return PT_OK;
}

void pt_destroy(pt_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* bufs[] = {c->d_samples, c->d_acc, c->d_cands, c->d_sse, c->d_gacc, c->d_bar,
                  c->d_err,     c->d_out, c->d_pop,   c->d_fit, c->d_u64};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

const char* pt_last_error(const pt_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pt_set_stream(pt_ctx* c, void* stream) {
  if (!c) return PT_EINVAL;
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return PT_OK;
}

void* pt_get_stream(const pt_ctx* c) { return c ? (void*)c->stream : nullptr; }

int pt_last_kernel_ms(const pt_ctx* c, float* ms) {
  if (!c || !ms) return PT_EINVAL;
  *ms = c->last_ms;
  return PT_OK;
}

int pt_load_block(pt_ctx* c, const void* samples, int64_t n, int dtype, double scale, double fs, double t0) {
  if (!c) return PT_EINVAL;
  const int es = esize_of(dtype);
  if (!samples || n < 1 || es == 0 || !(scale > 0.0) || !std::isfinite(scale) || !(fs > 0.0) ||
      !std::isfinite(fs) || !std::isfinite(t0))
    return fail(c, PT_EINVAL, "pt_load_block: invalid argument");
  if (n > (int64_t)1 << 36) return fail(c, PT_EINVAL, "pt_load_block: block too long");
  PT_CUDA(c, cudaSetDevice(c->device));
  c->has_block = false;
  const int64_t ntiles = (n + L - 1) / L;
  const size_t bytes = (size_t)ntiles * L * es;
  if (c->samples_cap < bytes) {
    if (c->d_samples) cudaFree(c->d_samples);
    c->d_samples = nullptr;
    c->samples_cap = 0;
    PT_CUDA(c, cudaMalloc(&c->d_samples, bytes));
    c->samples_cap = bytes;
  }
  const size_t nbytes = (size_t)n * es;
  PT_CUDA(c, cudaMemcpyAsync(c->d_samples, samples, nbytes, cudaMemcpyDefault, c->stream));
  if (bytes > nbytes)
    PT_CUDA(c, cudaMemsetAsync((char*)c->d_samples + nbytes, 0, bytes - nbytes, c->stream));
  PT_CUDA(c, cudaMemsetAsync(c->d_u64, 0, sizeof(unsigned long long), c->stream));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4LL * c->sms);
  k_absmax<<<grid, 256, 0, c->stream>>>(c->d_samples, n, dtype, c->d_u64);
  PT_CUDA(c, cudaGetLastError());
  unsigned long long bits = 0;
  PT_CUDA(c, cudaMemcpyAsync(&bits, c->d_u64, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(c, cudaStreamSynchronize(c->stream));
  double amax;
  std::memcpy(&amax, &bits, sizeof(amax));
  BlockArgs& b = c->blk;
  b.samples = c->d_samples;
  b.n = n;
  b.ntiles = ntiles;
  b.dtype = dtype;
  b.esize = es;
  b.scale = scale;
  b.smax = amax * scale;
  b.smax_f = (float)b.smax;
  if (!std::isfinite(b.smax)) return fail(c, PT_EINVAL, "pt_load_block: non-finite samples");
  b.t0 = t0;
  b.h = 1.0 / fs;
  b.t0sq_2 = t0 * t0 / 2.0;
  b.t0cu_6 = t0 * t0 * t0 / 6.0;
  b.h2_2 = b.h * b.h / 2.0;
  b.h3_6 = b.h * b.h * b.h / 6.0;
  c->has_block = true;
  return PT_OK;
}

int pt_objective(pt_ctx* c, const double* cands, int64_t n, double* sse_out, int tier) {
  if (!c) return PT_EINVAL;
  if (!cands || !sse_out || n < 1 || n > (1 << 24) || !valid_tier(tier))
    return fail(c, PT_EINVAL, "pt_objective: invalid argument");
  if (!c->has_block) return fail(c, PT_ENOBLOCK, "pt_objective: no block loaded");
  PT_CUDA(c, cudaSetDevice(c->device));
  int rc;
  if ((rc = ensure(c, &c->d_acc, &c->acc_cap, (size_t)n)) != PT_OK) return rc;
  if ((rc = ensure(c, &c->d_sse, &c->sse_cap, (size_t)n)) != PT_OK) return rc;
  const double* d_c = cands;
  if (!is_device_ptr(cands)) {
    if ((rc = ensure(c, &c->d_cands, &c->cands_cap, (size_t)n * D)) != PT_OK) return rc;
    PT_CUDA(c, cudaMemcpyAsync(c->d_cands, cands, (size_t)n * D * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream));
    d_c = c->d_cands;
  }
  const bool dev_out = is_device_ptr(sse_out);
  double* d_out = dev_out ? sse_out : c->d_sse;
  PT_CUDA(c, cudaMemsetAsync(c->d_acc, 0, (size_t)n * sizeof(unsigned long long), c->stream));
  PT_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  PT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  rc = launch_objective_any(c, tier, d_c, (int)n);
  if (rc != PT_OK) return rc;
  k_finalize<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(d_c, (int)n, c->d_acc, c->blk.n, c->blk.smax_f, d_out);
  PT_CUDA(c, cudaGetLastError());
  PT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  if (!dev_out)
    PT_CUDA(c, cudaMemcpyAsync(sse_out, d_out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if ((rc = kernel_error(c)) != PT_OK) return rc;
  PT_CUDA(c, cudaEventElapsedTime(&c->last_ms, c->ev0, c->ev1));
  return PT_OK;
}

int pt_de_solve_ex(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                   uint32_t block_id, double* params_out, double* pop_out, double* fit_out, int tier) {
  if (!c) return PT_EINVAL;
  if (!bounds || !params_out || pop < 4 || pop > PT_POP_MAX || gens < 0 || !valid_tier(tier) ||
      !std::isfinite(F) || !std::isfinite(CR) || CR < 0.0)
    return fail(c, PT_EINVAL, "pt_de_solve: invalid argument");
  if (is_device_ptr(bounds)) return fail(c, PT_EINVAL, "pt_de_solve: bounds must be a host pointer");
  for (int j = 0; j < D; ++j) {
    const double lo = bounds[2 * j], hi = bounds[2 * j + 1];
    if (!std::isfinite(lo) || !std::isfinite(hi) || lo > hi)
      return fail(c, PT_EINVAL, "pt_de_solve: bounds must be finite with lo <= hi");
  }
  if (!c->has_block) return fail(c, PT_ENOBLOCK, "pt_de_solve: no block loaded");
  PT_CUDA(c, cudaSetDevice(c->device));
  DeArgs a{};
  a.b = c->blk;
  for (int j = 0; j < D; ++j) {
    a.dc.lo[j] = bounds[2 * j];
    a.dc.hi[j] = bounds[2 * j + 1];
  }
  a.dc.F = F;
  a.dc.cr_all = CR >= 1.0;
  a.dc.cr_thr = CR >= 1.0 ? 0xffffffffu : (uint32_t)(CR * 4294967296.0);
  a.dc.periodic = (bounds[3] - bounds[2]) >= 2.0 * 3.14159265358979323846 * (1.0 - 1e-12);
  a.dc.key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  a.dc.block_id = block_id;
  a.np = pop;
  a.gens = gens;
  a.gacc = c->d_gacc;
  a.err = c->d_err;
  a.out = c->d_out;
  a.pop_out = c->d_pop;
  a.fit_out = c->d_fit;
  a.timeout_ns = c->timeout_ns;
  PT_CUDA(c, cudaMemsetAsync(c->d_gacc, 0, 3 * PT_POP_MAX * sizeof(unsigned long long), c->stream));
  PT_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  PT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  int rc = launch_de_any(c, tier, a);
  if (rc != PT_OK) return rc;
  PT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  if ((rc = kernel_error(c)) != PT_OK) return rc;
  PT_CUDA(c, cudaEventElapsedTime(&c->last_ms, c->ev0, c->ev1));
  PT_CUDA(c, cudaMemcpyAsync(params_out, c->d_out, (D + 1) * sizeof(double), cudaMemcpyDefault, c->stream));
  if (pop_out)
    PT_CUDA(c, cudaMemcpyAsync(pop_out, c->d_pop, (size_t)pop * D * sizeof(double), cudaMemcpyDefault, c->stream));
  if (fit_out)
    PT_CUDA(c, cudaMemcpyAsync(fit_out, c->d_fit, (size_t)pop * sizeof(double), cudaMemcpyDefault, c->stream));
  PT_CUDA(c, cudaStreamSynchronize(c->stream));
  return PT_OK;
}

int pt_de_solve(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                double* params_out, int tier) {
  return pt_de_solve_ex(c, bounds, pop, gens, F, CR, seed, 0u, params_out, nullptr, nullptr, tier);
}

}  // extern "C"
