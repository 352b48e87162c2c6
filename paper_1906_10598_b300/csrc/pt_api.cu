// C ABI of the phase-tracking hot path (declarations and contracts in
// include/phasetrack.h): contexts, block loading, the objective and the DE
// fit, plus the kernel launchers the batch and serving units share. Host side
// only validates arguments, sizes buffers and shapes launches; every step of
// the computation runs in the kernels of pt_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pt_grid.h"
#include "pt_internal.h"
#include "pt_kernels.cuh"

static_assert(pt::HOST_DE_GROUP_MAX == pt::DE_GROUP_MAX && pt::HOST_RING_SLOTS == pt::RING_SLOTS,
              "host mirrors of the DE group limit and ring depth");
static_assert(pt::HOST_NP_MAX == pt::NP_MAX && pt::HOST_RING_STRIDE == pt::RING_STRIDE && pt::HOST_L == pt::L &&
                  pt::HOST_D == pt::D && pt::HOST_DMAX == pt::DF && pt::HOST_MODEL_CUBIC == pt::MODEL_CUBIC &&
                  pt::HOST_MODEL_FULL == pt::MODEL_FULL,
              "host mirrors of the device constants");

namespace pt {

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

bool valid_tier(int t) { return t >= PT_TIER_F64 && t <= PT_TIER_F32; }

// Candidates per work item for the default tier: the width in {16, 8, 4}
// that pads `n` the least (wider on ties); the other tiers use 8.
int pick_cg(int tier, int n) { return tier == PT_TIER_F64 ? pick_cg_f64(n) : 8; }

namespace {

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

BlockArgs to_block_args(const HostBlock& h) {
  BlockArgs b{};
  b.samples = h.samples;
  b.n = h.n;
  b.ntiles = h.ntiles;
  b.dtype = h.dtype;
  b.esize = h.esize;
  b.scale = h.scale;
  b.smax = h.smax;
  b.smax_f = (float)h.smax;
  b.t0 = h.t0;
  b.h = 1.0 / h.fs;
  b.t0sq_2 = h.t0 * h.t0 / 2.0;
  b.t0cu_6 = h.t0 * h.t0 * h.t0 / 6.0;
  b.h2_2 = b.h * b.h / 2.0;
  b.h3_6 = b.h * b.h * b.h / 6.0;
  b.t0qu_24 = h.t0 * h.t0 * h.t0 * h.t0 / 24.0;
  b.h4_24 = b.h * b.h * b.h * b.h / 24.0;
  // quartic_needed: 2 pi ((M/2)^3 |S3| + (M/2)^4 |E4|), |S3| <= |E3| + 4 |E4| (n + 2 L), M/2 = 4
  b.quartic_k3 = 2.0 * 3.14159265358979323846 * 64.0;
  b.quartic_k4 = 2.0 * 3.14159265358979323846 * (256.0 + 4.0 * (double)(h.n + 2 * HOST_L) * 64.0);
  return b;
}

// ---- objective -------------------------------------------------------------

template <int TIER, int CGV, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC>
int launch_objective(pt_ctx* c, const double* d_cands, int ncand) {
  ObjArgs a{};
  a.b = to_block_args(c->blk);
  a.cands = d_cands;
  a.ncand = ncand;
  a.cpc = std::min(((ncand + CGV - 1) / CGV) * CGV, NP_MAX);
  const int ny = (ncand + a.cpc - 1) / a.cpc;
  // tiles split evenly, the grid sized to whole waves (objective_tiles_per_cta)
  a.tpc = objective_tiles_per_cta(a.b.ntiles, ny, OBJ_CTAS * c->sms, [&](int t) {
    return OBJ_CTAS * smem_layout(TIER, a.cpc, t, CGV, a.b.esize, 0, NT_OBJ, MODEL).total <= c->smem_optin;
  });
  const int nx = (int)((a.b.ntiles + a.tpc - 1) / a.tpc);
  a.acc = c->d_acc;
  a.err = c->d_err;
  a.timeout_ns = c->timeout_ns;
  a.extra_tx = c->inject_short_tx ? 16u : 0u;
  const SmemLayout S = smem_layout(TIER, a.cpc, a.tpc, CGV, a.b.esize, 0, NT_OBJ, MODEL);
  if (S.total > c->smem_optin) return fail(c, PT_EINVAL, "objective launch needs too much shared memory");
  PT_CUDA(c, cudaFuncSetAttribute(k_objective<TIER, CGV, OBJ, MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)S.total));
  dim3 grid(nx, ny);
  k_objective<TIER, CGV, OBJ, MODEL><<<grid, NT_OBJ, S.total, c->stream>>>(a);
  PT_CUDA(c, cudaGetLastError());
  return PT_OK;
}

int launch_objective_any(pt_ctx* c, int tier, const double* d_cands, int ncand, int model) {
  if (model == MODEL_FULL) {
    switch (tier) {
      case PT_TIER_F64: {
        const int cg = pick_cg(PT_TIER_F64, std::min(ncand, NP_MAX));
        if (cg == 16) return launch_objective<TIER_F64, 16, OBJ_CHI2, MODEL_FULL>(c, d_cands, ncand);
        if (cg == 8) return launch_objective<TIER_F64, 8, OBJ_CHI2, MODEL_FULL>(c, d_cands, ncand);
        return launch_objective<TIER_F64, 4, OBJ_CHI2, MODEL_FULL>(c, d_cands, ncand);
      }
      case PT_TIER_PLAIN: return launch_objective<TIER_PLAIN, 8, OBJ_CHI2, MODEL_FULL>(c, d_cands, ncand);
      case PT_TIER_DF32: return launch_objective<TIER_DF32, 8, OBJ_CHI2, MODEL_FULL>(c, d_cands, ncand);
      default: return launch_objective<TIER_F32, 8, OBJ_CHI2, MODEL_FULL>(c, d_cands, ncand);
    }
  }
  if (c->objective == PT_OBJ_COR) {
    switch (tier) {
      case PT_TIER_F64: {
        const int cg = pick_cg(tier, std::min(ncand, NP_MAX));
        if (cg == 16) return launch_objective<TIER_F64, 16, OBJ_COR>(c, d_cands, ncand);
        if (cg == 8) return launch_objective<TIER_F64, 8, OBJ_COR>(c, d_cands, ncand);
        return launch_objective<TIER_F64, 4, OBJ_COR>(c, d_cands, ncand);
      }
      case PT_TIER_PLAIN: return launch_objective<TIER_PLAIN, 8, OBJ_COR>(c, d_cands, ncand);
      case PT_TIER_DF32: return launch_objective<TIER_DF32, 8, OBJ_COR>(c, d_cands, ncand);
      default: return launch_objective<TIER_F32, 8, OBJ_COR>(c, d_cands, ncand);
    }
  }
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

// ---- grouped DE --------------------------------------------------------------

size_t smem_de(int tier, int sc_tiles, int esize_max, int model, bool ahead) {
  return smem_layout(tier, NP_MAX, sc_tiles, 16, esize_max, NP_MAX, NT, model, ahead).total;
}

template <int TIER, int OBJ = OBJ_CHI2, int MODEL = MODEL_CUBIC, int SK = -1, int CGK = 0>
int launch_de_t(pt_ctx* c, cudaStream_t s, DeLaunch& a) {
  const size_t smem = smem_de(TIER, a.sc_tiles, a.esize_max, MODEL, a.ahead != 0);
  cudaFuncAttributes fa{};
  PT_CUDA(c, cudaFuncGetAttributes(&fa, k_de<TIER, OBJ, MODEL, SK, CGK>));
  if (smem + fa.sharedSizeBytes > c->smem_optin) return fail(c, PT_EINVAL, "DE launch needs too much shared memory");
  PT_CUDA(c, cudaFuncSetAttribute(k_de<TIER, OBJ, MODEL, SK, CGK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  PT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_de<TIER, OBJ, MODEL, SK, CGK>, NT, smem));
  // pt_inject_missing_cta: the last group's last rank is not started, so its
  // arrivals never come and the others' bounded waits run out
  const int grid = a.ngroups * a.k - (c->inject_missing_cta && a.ngroups * a.k > 1 ? 1 : 0);
  if (occ < 1 || grid > occ * c->sms) return fail(c, PT_EINVAL, "DE grid cannot be co-resident");
  void* args[] = {&a};
  PT_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_de<TIER, OBJ, MODEL, SK, CGK>, dim3(grid), dim3(NT), args, smem, s));
  return PT_OK;
}

// The default tier's DE kernels are compiled per strategy (every block of a
// launch has the context's strategy), and once more for launches whose blocks
// all evaluate 16-candidate items on resident tiles (cg16 and a.ahead).
template <int OBJ, int MODEL = MODEL_CUBIC>
int launch_de_f64(pt_ctx* c, cudaStream_t s, DeLaunch& a, bool cg16) {
  if (cg16 && a.ahead) {
    switch (c->strategy) {
      case DE_BEST1_JITTER: return launch_de_t<TIER_F64, OBJ, MODEL, DE_BEST1_JITTER, 16>(c, s, a);
      case DE_EITHER_OR: return launch_de_t<TIER_F64, OBJ, MODEL, DE_EITHER_OR, 16>(c, s, a);
      default: return launch_de_t<TIER_F64, OBJ, MODEL, DE_RAND1_BIN, 16>(c, s, a);
    }
  }
  switch (c->strategy) {
    case DE_BEST1_JITTER: return launch_de_t<TIER_F64, OBJ, MODEL, DE_BEST1_JITTER>(c, s, a);
    case DE_EITHER_OR: return launch_de_t<TIER_F64, OBJ, MODEL, DE_EITHER_OR>(c, s, a);
    default: return launch_de_t<TIER_F64, OBJ, MODEL, DE_RAND1_BIN>(c, s, a);
  }
}

// Device layout of the descriptor buffer: blocks | sched | sched_off.
size_t o_sched(int nblocks) { return align_up((size_t)nblocks * sizeof(DeBlockDesc), 256); }
size_t o_off(int nblocks) { return o_sched(nblocks) + align_up((size_t)nblocks * sizeof(int), 256); }

}  // namespace

size_t de_desc_bytes(int nblocks, int ngroups) { return o_off(nblocks) + (size_t)(ngroups + 1) * sizeof(int); }

// The DE kernel's static shared memory (its block descriptor and a few flags,
// under 1 KB) comes out of the same per-block opt-in budget as the dynamic part.
constexpr size_t DE_STATIC_SMEM_RESERVE = 2048;

int pick_sc_tiles(pt_ctx* c, int tier, int esize_max, int64_t want, int model, bool ahead) {
  int sc = (int)std::max<int64_t>(1, std::min<int64_t>(want, 96));
  while (sc > 1 && smem_de(tier, sc, esize_max, model, ahead) + DE_STATIC_SMEM_RESERVE > c->smem_optin) sc--;
  return sc;
}

int load_samples(pt_ctx* c, cudaStream_t s, const void* samples, int64_t n, int dtype, double scale, double fs,
                 double t0, void** dbuf, size_t* cap, unsigned long long* d_u64, HostBlock* hb) {
  const int es = esize_of(dtype);
  if (!samples || n < 1 || es == 0 || !(scale > 0.0) || !std::isfinite(scale) || !(fs > 0.0) ||
      !std::isfinite(fs) || !std::isfinite(t0))
    return fail(c, PT_EINVAL, "load: invalid argument");
  if (n > (int64_t)1 << 36) return fail(c, PT_EINVAL, "load: block too long");
  const int64_t ntiles = (n + L - 1) / L;
  const size_t bytes = (size_t)ntiles * L * es;
  if (*cap < bytes) {
    if (*dbuf) cudaFree(*dbuf);
    *dbuf = nullptr;
    *cap = 0;
    PT_CUDA(c, cudaMalloc(dbuf, bytes));
    *cap = bytes;
  }
  const size_t nbytes = (size_t)n * es;
  PT_CUDA(c, cudaMemcpyAsync(*dbuf, samples, nbytes, cudaMemcpyDefault, s));
  if (bytes > nbytes) PT_CUDA(c, cudaMemsetAsync((char*)*dbuf + nbytes, 0, bytes - nbytes, s));
  PT_CUDA(c, cudaMemsetAsync(d_u64, 0, sizeof(unsigned long long), s));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4LL * c->sms);
  k_absmax<<<grid, 256, 0, s>>>(*dbuf, n, dtype, d_u64);
  PT_CUDA(c, cudaGetLastError());
  unsigned long long bits = 0;
  PT_CUDA(c, cudaMemcpyAsync(&bits, d_u64, sizeof(bits), cudaMemcpyDeviceToHost, s));
  PT_CUDA(c, cudaStreamSynchronize(s));
  double amax;
  std::memcpy(&amax, &bits, sizeof(amax));
  hb->samples = *dbuf;
  hb->n = n;
  hb->ntiles = ntiles;
  hb->dtype = dtype;
  hb->esize = es;
  hb->scale = scale;
  hb->smax = amax * scale;
  hb->t0 = t0;
  hb->fs = fs;
  if (!std::isfinite(hb->smax)) return fail(c, PT_EINVAL, "load: non-finite samples");
  return PT_OK;
}

int check_de_args(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, int tier, int dim) {
  if (!bounds || pop < 4 || pop > PT_POP_MAX || gens < 0 || !valid_tier(tier) || !std::isfinite(F) ||
      !std::isfinite(CR) || CR < 0.0)
    return fail(c, PT_EINVAL, "DE: invalid argument");
  if (is_device_ptr(bounds)) return fail(c, PT_EINVAL, "DE: bounds must be a host pointer");
  for (int j = 0; j < dim; ++j) {
    const double lo = bounds[2 * j], hi = bounds[2 * j + 1];
    if (!std::isfinite(lo) || !std::isfinite(hi) || lo > hi)
      return fail(c, PT_EINVAL, "DE: bounds must be finite with lo <= hi");
  }
  return PT_OK;
}

}  // namespace pt

namespace pt {

int launch_de_groups(pt_ctx* c, cudaStream_t s, int tier, const HostDeBlock* blocks, int nblocks, const int* sched,
                     const int* off, int ngroups, int k, void* d_desc_buf, unsigned long long* ring, int* d_err,
                     int mode, int model) {
  // the arrival count of a ring word is its low byte (de_block): k <= 255
  if (k < 1 || k > HOST_DE_GROUP_MAX) return fail(c, PT_EINVAL, "DE group size must be 1 .. 255 CTAs");
  std::vector<DeBlockDesc> desc(nblocks);
  bool cg16 = true;  // every block evaluates 16-candidate items
  int esize_max = 1;
  int64_t want = 1;
  for (int i = 0; i < nblocks; ++i) {
    const HostDeBlock& h = blocks[i];
    DeBlockDesc& d = desc[i];
    d.b = to_block_args(h.blk);
    for (int j = 0; j < DF; ++j) {
      d.dc.lo[j] = j < model_dim(model) ? h.lo[j] : 0.0;
      d.dc.hi[j] = j < model_dim(model) ? h.hi[j] : 0.0;
    }
    d.dc.F = h.F;
    d.dc.K = (h.F + 1.0) * 0.5;
    d.dc.strategy = c->strategy;
    d.dc.cr_all = h.CR >= 1.0;
    d.dc.cr_thr = h.CR >= 1.0 ? 0xffffffffu : (uint32_t)(h.CR * 4294967296.0);
    d.dc.periodic = (h.hi[1] - h.lo[1]) >= 2.0 * 3.14159265358979323846 * (1.0 - 1e-12);
    d.dc.key = make_uint2((uint32_t)(h.seed & 0xffffffffu), (uint32_t)(h.seed >> 32));
    d.dc.block_id = h.block_id;
    d.np = h.pop;
    d.gens = h.gens;
    d.cg = pick_cg(tier, h.pop);
    cg16 = cg16 && d.cg == 16;
    d.out = h.out;
    d.pop_out = h.pop_out;
    d.fit_out = h.fit_out;
    esize_max = std::max(esize_max, h.blk.esize);
    // a CTA's share of items spans at most one tile more than ntiles / k
    want = std::max<int64_t>(want, std::min<int64_t>(h.blk.ntiles, (h.blk.ntiles + k - 1) / k + 1));
  }
  char* base = (char*)d_desc_buf;
  if (mode & DE_UPLOAD) {
    // pageable sources: each copy has consumed its source when it returns
    PT_CUDA(c, cudaMemcpyAsync(base, desc.data(), nblocks * sizeof(DeBlockDesc), cudaMemcpyHostToDevice, s));
    PT_CUDA(c, cudaMemcpyAsync(base + o_sched(nblocks), sched, nblocks * sizeof(int), cudaMemcpyHostToDevice, s));
    PT_CUDA(c, cudaMemcpyAsync(base + o_off(nblocks), off, (ngroups + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  DeLaunch a{};
  a.blocks = (const DeBlockDesc*)base;
  a.sched = (const int*)(base + o_sched(nblocks));
  a.sched_off = (const int*)(base + o_off(nblocks));
  a.ngroups = ngroups;
  a.k = k;
  // the next generation is built ahead only on resident tiles, so its second
  // trial set is laid out only when every block's share fits beside it; else
  // the staging chunk gets that shared memory
  a.sc_tiles = pick_sc_tiles(c, tier, esize_max, want, model, true);
  a.ahead = a.sc_tiles >= want ? 1 : 0;
  if (!a.ahead) a.sc_tiles = pick_sc_tiles(c, tier, esize_max, want, model, false);
  a.esize_max = esize_max;
  a.ring = ring;
  a.err = d_err;
  a.timeout_ns = c->timeout_ns;
  a.extra_tx = c->inject_short_tx ? 16u : 0u;
  if (!(mode & DE_LAUNCH)) return PT_OK;
  PT_CUDA(c, cudaMemsetAsync(ring, 0, (size_t)ngroups * RING_GROUP_WORDS * sizeof(unsigned long long), s));
  PT_CUDA(c, cudaMemsetAsync(d_err, 0, sizeof(int), s));
  if (model == MODEL_FULL) {
    // the full model: the chi-square (checked by the entry points)
    a.obj = OBJ_CHI2;
    switch (tier) {
      case PT_TIER_F64: return launch_de_f64<OBJ_CHI2, MODEL_FULL>(c, s, a, cg16);
      case PT_TIER_PLAIN: return launch_de_t<TIER_PLAIN, OBJ_CHI2, MODEL_FULL>(c, s, a);
      case PT_TIER_DF32: return launch_de_t<TIER_DF32, OBJ_CHI2, MODEL_FULL>(c, s, a);
      default: return launch_de_t<TIER_F32, OBJ_CHI2, MODEL_FULL>(c, s, a);
    }
  }
  a.obj = c->objective;
  if (a.obj == OBJ_COR) {
    switch (tier) {
      case PT_TIER_F64: return launch_de_f64<OBJ_COR>(c, s, a, cg16);
      case PT_TIER_PLAIN: return launch_de_t<TIER_PLAIN, OBJ_COR>(c, s, a);
      case PT_TIER_DF32: return launch_de_t<TIER_DF32, OBJ_COR>(c, s, a);
      default: return launch_de_t<TIER_F32, OBJ_COR>(c, s, a);
    }
  }
  switch (tier) {
    case PT_TIER_F64: return launch_de_f64<OBJ_CHI2>(c, s, a, cg16);
    case PT_TIER_PLAIN: return launch_de_t<TIER_PLAIN>(c, s, a);
    case PT_TIER_DF32: return launch_de_t<TIER_DF32>(c, s, a);
    default: return launch_de_t<TIER_F32>(c, s, a);
  }
}

int launch_absmax(pt_ctx* c, cudaStream_t s, const void* dsamples, int64_t n, int dtype, unsigned long long* d_slot) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4LL * c->sms));
  k_absmax<<<grid, 256, 0, s>>>(dsamples, n, dtype, d_slot);
  PT_CUDA(c, cudaGetLastError());
  return PT_OK;
}

int kernel_status(pt_ctx* c, cudaStream_t s, int* d_err) {
  int h_err = 0;
  PT_CUDA(c, cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PT_CUDA(c, cudaStreamSynchronize(s));
  if (h_err == DEV_TIMEOUT) return fail(c, PT_ETIMEOUT, "a bounded device-side wait expired");
  if (h_err != DEV_OK) return fail(c, PT_ECUDA, "device error status " + std::to_string(h_err));
  return PT_OK;
}

}  // namespace pt

using namespace pt;

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
  if (bad(cudaMalloc(&c->d_ring, (size_t)c->sms * RING_GROUP_WORDS * sizeof(unsigned long long)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_err, sizeof(int)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_out, 8 * sizeof(double)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_pop, PT_POP_MAX * DF * sizeof(double)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_fit, PT_POP_MAX * sizeof(double)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_u64, sizeof(unsigned long long)))) return PT_ENOMEM;
  if (bad(cudaMalloc(&c->d_desc, de_desc_bytes(1, 1)))) return PT_ENOMEM;
  if (bad(cudaEventCreate(&c->ev0))) return PT_ECUDA;
  if (bad(cudaEventCreate(&c->ev1))) return PT_ECUDA;
  *out = c;
  return PT_OK;
}

void pt_serve_shutdown(pt_ctx* c);  // pt_serve.cu

void pt_destroy(pt_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  pt_serve_shutdown(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* bufs[] = {c->d_samples, c->d_acc, c->d_cands, c->d_sse, c->d_ring, c->d_err,
                  c->d_out,     c->d_pop, c->d_fit,   c->d_u64, c->d_desc, c->d_seed};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

const char* pt_last_error(const pt_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pt_set_strategy(pt_ctx* c, int strategy) {
  if (!c) return PT_EINVAL;
  if (strategy != PT_DE_RAND1_BIN && strategy != PT_DE_BEST1_JITTER && strategy != PT_DE_EITHER_OR)
    return fail(c, PT_EINVAL, "unknown DE strategy");
  c->strategy = strategy;
  return PT_OK;
}

int pt_set_wait_timeout(pt_ctx* c, double seconds) {
  if (!c) return PT_EINVAL;
  if (!(seconds >= 1e-3 && seconds <= 60.0)) return fail(c, PT_EINVAL, "pt_set_wait_timeout: 1e-3 .. 60 s");
  c->timeout_ns = (uint64_t)(seconds * 1e9);
  return PT_OK;
}

int pt_inject_missing_cta(pt_ctx* c, int enable) {
  if (!c) return PT_EINVAL;
  c->inject_missing_cta = enable != 0;
  return PT_OK;
}

int pt_inject_short_tx(pt_ctx* c, int enable) {
  if (!c) return PT_EINVAL;
  c->inject_short_tx = enable != 0;
  return PT_OK;
}

int pt_set_objective(pt_ctx* c, int objective) {
  if (!c) return PT_EINVAL;
  if (objective != PT_OBJ_CHI2 && objective != PT_OBJ_COR) return fail(c, PT_EINVAL, "unknown objective");
  c->objective = objective;
  return PT_OK;
}

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
  PT_CUDA(c, cudaSetDevice(c->device));
  c->has_block = false;
  const int rc = load_samples(c, c->stream, samples, n, dtype, scale, fs, t0, &c->d_samples, &c->samples_cap,
                              c->d_u64, &c->blk);
  if (rc != PT_OK) return rc;
  c->has_block = true;
  return PT_OK;
}

}  // extern "C"

namespace {

// pt_objective / pt_objective_full: candidates of model_dim(model) parameters.
int objective_impl(pt_ctx* c, const double* cands, int64_t n, double* sse_out, int tier, int model) {
  const int dim = model_dim(model);
  if (!cands || !sse_out || n < 1 || n > (1 << 24) || !valid_tier(tier))
    return fail(c, PT_EINVAL, "pt_objective: invalid argument");
  if (!c->has_block) return fail(c, PT_ENOBLOCK, "pt_objective: no block loaded");
  PT_CUDA(c, cudaSetDevice(c->device));
  int rc;
  if ((rc = ensure(c, &c->d_acc, &c->acc_cap, (size_t)n)) != PT_OK) return rc;
  if ((rc = ensure(c, &c->d_sse, &c->sse_cap, (size_t)n)) != PT_OK) return rc;
  const double* d_c = cands;
  if (!is_device_ptr(cands)) {
    if ((rc = ensure(c, &c->d_cands, &c->cands_cap, (size_t)n * dim)) != PT_OK) return rc;
    PT_CUDA(c, cudaMemcpyAsync(c->d_cands, cands, (size_t)n * dim * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream));
    d_c = c->d_cands;
  }
  const bool dev_out = is_device_ptr(sse_out);
  double* d_out = dev_out ? sse_out : c->d_sse;
  PT_CUDA(c, cudaMemsetAsync(c->d_acc, 0, (size_t)n * sizeof(unsigned long long), c->stream));
  PT_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  PT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  rc = launch_objective_any(c, tier, d_c, (int)n, model);
  if (rc != PT_OK) return rc;
  k_finalize<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(d_c, (int)n, c->d_acc, c->blk.n, (float)c->blk.smax,
                                                             d_out, c->objective, model, c->blk.t0,
                                                             1.0 / c->blk.fs);
  PT_CUDA(c, cudaGetLastError());
  PT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  if (!dev_out)
    PT_CUDA(c, cudaMemcpyAsync(sse_out, d_out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if ((rc = kernel_status(c, c->stream, c->d_err)) != PT_OK) return rc;
  PT_CUDA(c, cudaEventElapsedTime(&c->last_ms, c->ev0, c->ev1));
  return PT_OK;
}

// pt_de_solve_ex / pt_de_solve_full: bounds, params_out and pop_out of
// model_dim(model) parameters.
int de_solve_impl(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                  uint32_t block_id, double* params_out, double* pop_out, double* fit_out, int tier, int model) {
  const int dim = model_dim(model);
  int rc = check_de_args(c, bounds, pop, gens, F, CR, tier, dim);
  if (rc != PT_OK) return rc;
  if (!params_out) return fail(c, PT_EINVAL, "pt_de_solve: params_out is null");
  if (!c->has_block) return fail(c, PT_ENOBLOCK, "pt_de_solve: no block loaded");
  PT_CUDA(c, cudaSetDevice(c->device));
  HostDeBlock h;
  h.blk = c->blk;
  for (int j = 0; j < dim; ++j) {
    h.lo[j] = bounds[2 * j];
    h.hi[j] = bounds[2 * j + 1];
  }
  h.pop = pop;
  h.gens = gens;
  h.F = F;
  h.CR = CR;
  h.seed = seed;
  h.block_id = block_id;
  h.out = c->d_out;
  h.pop_out = c->d_pop;
  h.fit_out = c->d_fit;
  const int sched[1] = {0}, off[2] = {0, 1};
  const int k = (int)std::min<int64_t>(std::min<int64_t>(c->blk.ntiles, c->sms), HOST_DE_GROUP_MAX);
  PT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  rc = launch_de_groups(c, c->stream, tier, &h, 1, sched, off, 1, k, c->d_desc, c->d_ring, c->d_err,
                        DE_UPLOAD | DE_LAUNCH, model);
  if (rc != PT_OK) return rc;
  PT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  if ((rc = kernel_status(c, c->stream, c->d_err)) != PT_OK) return rc;
  PT_CUDA(c, cudaEventElapsedTime(&c->last_ms, c->ev0, c->ev1));
  PT_CUDA(c, cudaMemcpyAsync(params_out, c->d_out, (dim + 1) * sizeof(double), cudaMemcpyDefault, c->stream));
  if (pop_out)
    PT_CUDA(c, cudaMemcpyAsync(pop_out, c->d_pop, (size_t)pop * dim * sizeof(double), cudaMemcpyDefault, c->stream));
  if (fit_out)
    PT_CUDA(c, cudaMemcpyAsync(fit_out, c->d_fit, (size_t)pop * sizeof(double), cudaMemcpyDefault, c->stream));
  PT_CUDA(c, cudaStreamSynchronize(c->stream));
  return PT_OK;
}

// The full model runs on the chi-square only (Eq. 2-2-5's model has a
// constant amplitude); every tier and DE strategy applies.
int check_full_settings(pt_ctx* c) {
  if (c->objective != PT_OBJ_CHI2)
    return fail(c, PT_EINVAL, "the full model runs on the chi-square objective only");
  return PT_OK;
}

}  // namespace

extern "C" {

int pt_objective(pt_ctx* c, const double* cands, int64_t n, double* sse_out, int tier) {
  if (!c) return PT_EINVAL;
  return objective_impl(c, cands, n, sse_out, tier, MODEL_CUBIC);
}

int pt_objective_full(pt_ctx* c, const double* cands, int64_t n, double* sse_out, int tier) {
  if (!c) return PT_EINVAL;
  const int rc = check_full_settings(c);
  if (rc != PT_OK) return rc;
  return objective_impl(c, cands, n, sse_out, tier, MODEL_FULL);
}

int pt_de_solve_ex(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                   uint32_t block_id, double* params_out, double* pop_out, double* fit_out, int tier) {
  if (!c) return PT_EINVAL;
  return de_solve_impl(c, bounds, pop, gens, F, CR, seed, block_id, params_out, pop_out, fit_out, tier, MODEL_CUBIC);
}

int pt_de_solve_full(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                     uint32_t block_id, double* params_out, double* pop_out, double* fit_out, int tier) {
  if (!c) return PT_EINVAL;
  const int rc = check_full_settings(c);
  if (rc != PT_OK) return rc;
  return de_solve_impl(c, bounds, pop, gens, F, CR, seed, block_id, params_out, pop_out, fit_out, tier, MODEL_FULL);
}

int pt_de_solve(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                double* params_out, int tier) {
  return pt_de_solve_ex(c, bounds, pop, gens, F, CR, seed, 0u, params_out, nullptr, nullptr, tier);
}

}  // extern "C"
