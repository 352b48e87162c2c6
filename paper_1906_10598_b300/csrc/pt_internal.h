// Host-side internals shared by the translation units of libphasetrack:
// the context, error helpers and the launchers of the device kernels.
// Not part of the public ABI (include/phasetrack.h).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <memory>
#include <string>

#include "../../include/phasetrack.h"

struct pt_serve_state;  // serving scheduler (pt_serve.cu)

namespace pt {

// Mirrors of the device-side descriptors (pt_kernels.cuh) that host code
// needs to size buffers; the launchers below fill the real structs.
constexpr int HOST_L = 256;      // samples per tile
constexpr int HOST_D = 5;        // parameters per candidate
constexpr int HOST_DMAX = 7;     // parameters per candidate of the full model
constexpr int HOST_MODEL_CUBIC = 0, HOST_MODEL_FULL = 1;
constexpr int HOST_NP_MAX = 128;
constexpr int HOST_RING_STRIDE = 16;  // 64-bit words per candidate slot of the DE exchange ring
// Largest DE group (CTAs solving one block together): each exchange word
// counts the group's arrivals in its low byte (k_de's ring, pt_kernels.cuh),
// so a group of 256 or more CTAs would carry into the sum.
constexpr int HOST_DE_GROUP_MAX = 255;
// words of one group's DE exchange ring: HOST_RING_SLOTS generations x HOST_NP_MAX candidates
constexpr int HOST_RING_SLOTS = 4;
constexpr size_t RING_GROUP_WORDS = (size_t)HOST_RING_SLOTS * HOST_NP_MAX * HOST_RING_STRIDE;

// Per-block constants computed at load time (same meaning as BlockArgs).
struct HostBlock {
  const void* samples = nullptr;  // device, zero-padded to a multiple of HOST_L samples
  int64_t n = 0;
  int64_t ntiles = 0;
  int dtype = 0;
  int esize = 0;
  double scale = 1.0;
  double smax = 0.0;
  double t0 = 0.0, fs = 1.0;
};

// One DE problem as the host describes it to the grouped launcher.
struct HostDeBlock {
  HostBlock blk;
  double lo[HOST_DMAX], hi[HOST_DMAX];  // the model's first 5 or 7 used
  int pop = 0, gens = 0;
  double F = 0.7, CR = 0.9;
  uint64_t seed = 0;
  uint32_t block_id = 0;
  double* out = nullptr;      // device [dim + 1]
  double* pop_out = nullptr;  // device [pop*dim] or null
  double* fit_out = nullptr;  // device [pop] or null
};

}  // namespace pt

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
  pt::HostBlock blk;
  bool has_block = false;
  // objective scratch
  unsigned long long* d_acc = nullptr;
  size_t acc_cap = 0;
  double* d_cands = nullptr;
  size_t cands_cap = 0;
  double* d_sse = nullptr;
  size_t sse_cap = 0;
  // DE scratch: rings for up to `sms` groups, results of one block
  unsigned long long* d_ring = nullptr;
  int* d_err = nullptr;
  double* d_out = nullptr;
  double* d_pop = nullptr;
  double* d_fit = nullptr;
  unsigned long long* d_u64 = nullptr;
  void* d_desc = nullptr;  // one block descriptor + a one-entry schedule
  void* d_seed = nullptr;  // pt_seed_bounds: three peaks and the result
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  float last_ms = 0.f;
  uint64_t timeout_ns = 2000000000ull;
  bool inject_missing_cta = false;  // pt_inject_missing_cta (tests of the bounded waits)
  bool inject_short_tx = false;     // pt_inject_short_tx (test of the staging wait's limit)
  int objective = 0;  // PT_OBJ_CHI2 or PT_OBJ_COR, for pt_objective and the DE entry points
  int strategy = 0;   // PT_DE_*, for the DE entry points
  // autotune cache of the batched launcher: per-CTA rate and per-generation costs
  double tune_rate = 0.0, tune_fixed_s = 0.0;
  double tune_rate_stream = 0.0;  // per-CTA rate when a CTA's tiles are staged chunk by chunk
  int tune_res_tiles = 0;         // tiles one CTA keeps resident (its shared-memory capacity)
  int tune_model = 0;             // the model the cached rates were measured on
  bool tuned = false;
  pt_serve_state* serve = nullptr;
};

namespace pt {

inline int fail(pt_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define PT_CUDA(ctx, call)                                                                      \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      return ::pt::fail(ctx, e_ == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    }                                                                                           \
  } while (0)

bool is_device_ptr(const void* p);
int esize_of(int dtype);
bool valid_tier(int t);
int pick_cg(int tier, int n);

// Copy `n` samples (host or device) into `*dbuf` (grown as needed, padded with
// zeros to a multiple of HOST_L) on `stream`, measure max |sample| with a
// kernel, and fill `hb`. Synchronises `stream`.
int load_samples(pt_ctx* c, cudaStream_t stream, const void* samples, int64_t n, int dtype, double scale, double fs,
                 double t0, void** dbuf, size_t* cap, unsigned long long* d_u64, HostBlock* hb);

// Validate DE arguments (bounds host pointer, dim x 2).
int check_de_args(pt_ctx* c, const double* bounds, int pop, int gens, double F, double CR, int tier,
                  int dim = HOST_D);

// Launch the grouped persistent DE kernel: `ngroups` groups of `k` CTAs,
// group q solving blocks sched[off[q] .. off[q+1]) of `blocks` (host array,
// uploaded into `d_desc_buf`, which must hold nblocks descriptors plus the
// schedule; `mode` says whether to upload them from host memory, to launch,
// or both). `ring` holds ngroups * RING_GROUP_WORDS words; ring and *d_err
// are cleared on `stream` first. Asynchronous.
constexpr int DE_UPLOAD = 1;  // copy descriptors and schedule to d_desc_buf
constexpr int DE_LAUNCH = 2;  // clear ring and error word, launch
int launch_de_groups(pt_ctx* c, cudaStream_t stream, int tier, const HostDeBlock* blocks, int nblocks,
                     const int* sched, const int* off, int ngroups, int k, void* d_desc_buf,
                     unsigned long long* ring, int* d_err, int mode, int model = HOST_MODEL_CUBIC);

// max |stored sample| of n samples at dsamples into *d_slot (which must be
// zeroed first) by the absmax kernel. Asynchronous.
int launch_absmax(pt_ctx* c, cudaStream_t s, const void* dsamples, int64_t n, int dtype, unsigned long long* d_slot);

// Read a launch's device error word (synchronises `s`).
int kernel_status(pt_ctx* c, cudaStream_t s, int* d_err);

// Bytes of device memory launch_de_groups needs for its descriptors.
size_t de_desc_bytes(int nblocks, int ngroups);

// Staged tiles per CTA for a launch whose CTAs own at most `want` tiles.
int pick_sc_tiles(pt_ctx* c, int tier, int esize_max, int64_t want, int model = HOST_MODEL_CUBIC,
                  bool ahead = true);

}  // namespace pt
