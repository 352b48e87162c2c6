// Batched DE fits (pt_batch_*): many independent blocks, one persistent
// cooperative launch over groups of CTAs, replayed from a captured CUDA graph.
//
// Autotuner: the per-generation time of one block on k CTAs is modelled as
//   t(k) = ceil(ntiles / k) * 256 * npad / R + c_gen,
// with R the objective rate of one CTA (R_res while a CTA's tiles fit its
// shared memory, R_stream when they are staged chunk by chunk each
// generation) and c_gen the fixed per-generation cost (trial generation, FP64
// set-up, exchange, selection). R_res and c_gen come from short DE runs of the
// batch's first block at its own population on two group sizes that keep the
// tiles resident (the work per CTA differs, nothing else); R_stream from a
// third run with about three times the resident capacity per CTA, when the
// block is that large. They are cached in the context. For each candidate group
// size k the blocks are assigned longest-first to the least-loaded of the
// floor(SMs / k) groups (LPT); the k with the shortest predicted makespan wins.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "pt_internal.h"

using namespace pt;

struct pt_batch {
  pt_ctx* ctx = nullptr;
  int tier = 0;
  int model = HOST_MODEL_CUBIC;     // HOST_MODEL_FULL: pt_batch_create_full
  int dim = HOST_D;                 // parameters per block fit
  int nblocks = 0;
  int ngroups = 0, k = 0;
  double predicted_ms = 0.0, sample_evals = 0.0;
  float last_ms = 0.f;
  void* d_arena = nullptr;          // all blocks' samples, each padded to a whole tile
  unsigned long long* d_amax = nullptr;
  double* d_out = nullptr;          // nblocks x (dim + 1)
  void* d_desc = nullptr;           // descriptors + schedule
  unsigned long long* d_ring = nullptr;
  int* d_err = nullptr;
  std::vector<HostDeBlock> blocks;
  std::vector<int> sched, off;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int64_t padded_bytes(int64_t n, int esize) { return (n + HOST_L - 1) / HOST_L * HOST_L * esize; }

// Per-generation seconds of one DE run of `b` on k CTAs: time two runs that
// differ only in the generation count and difference them.
int time_per_gen(pt_ctx* c, int tier, HostDeBlock b, int k, int model, double* out) {
  const int sched[1] = {0}, off[2] = {0, 1};
  float ms[2];
  const int gens[2] = {4, 16};
  for (int r = 0; r < 2; ++r) {
    b.gens = gens[r];
    b.out = c->d_out;
    b.pop_out = nullptr;
    b.fit_out = nullptr;
    PT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
    int rc = launch_de_groups(c, c->stream, tier, &b, 1, sched, off, 1, k, c->d_desc, c->d_ring, c->d_err,
                              DE_UPLOAD | DE_LAUNCH, model);
    if (rc != PT_OK) return rc;
    PT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
    if ((rc = kernel_status(c, c->stream, c->d_err)) != PT_OK) return rc;
    PT_CUDA(c, cudaEventElapsedTime(&ms[r], c->ev0, c->ev1));
  }
  *out = std::max(1e-9, (ms[1] - ms[0]) * 1e-3 / (gens[1] - gens[0]));
  return PT_OK;
}

int npad_of(int tier, int pop) {
  const int cg = pick_cg(tier, pop);
  return (pop + cg - 1) / cg * cg;
}

// Samples one CTA of a group of k evaluates per generation.
double cta_samples(int64_t ntiles, int k) { return (double)((ntiles + k - 1) / k) * HOST_L; }

// Whether one CTA of a group of k keeps its share of the block resident (its
// item share spans at most one tile more than ntiles / k).
bool resident(const pt_ctx* c, int64_t ntiles, int k) { return (ntiles + k - 1) / k + 1 <= c->tune_res_tiles; }

int clamp_k(const pt_ctx* c, int64_t k) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(k, std::min(c->sms, HOST_DE_GROUP_MAX)));
}

// Calibrate R_res, R_stream and c_gen (cached in the context for the model
// they were measured on).
int calibrate(pt_ctx* c, int tier, const HostDeBlock& b0, int model) {
  if (c->tuned && c->tune_model == model) return PT_OK;
  const HostDeBlock& b = b0;
  const int64_t nt = b.blk.ntiles;
  const double np = (double)npad_of(tier, b.pop);
  // the most tiles a CTA keeps resident (without the second trial set)
  const int S = pick_sc_tiles(c, tier, b.blk.esize, 96, model, false);
  c->tune_res_tiles = S;
  // two resident shapes: about S/3 and 2S/3 tiles per CTA
  int ka = clamp_k(c, (nt + std::max(1, S / 3) - 1) / std::max(1, S / 3));
  int kb = clamp_k(c, (nt + std::max(1, 2 * S / 3) - 1) / std::max(1, 2 * S / 3));
  if (kb >= ka) kb = std::max(1, ka / 2);
  double ta, tb;
  int rc;
  // the context's first DE launch also loads the module: run one untimed first
  if ((rc = time_per_gen(c, tier, b, ka, model, &ta)) != PT_OK) return rc;
  if ((rc = time_per_gen(c, tier, b, ka, model, &ta)) != PT_OK) return rc;
  if ((rc = time_per_gen(c, tier, b, kb, model, &tb)) != PT_OK) return rc;
  const double wa = cta_samples(nt, ka), wb = cta_samples(nt, kb);
  const double R = (wb > wa && tb > ta) ? (wb - wa) * np / (tb - ta) : wa * np / ta;
  const double cg = std::max(0.0, ta - wa * np / R);
  double Rs = R;
  if (nt >= 3 * (int64_t)S) {
    const int ks = clamp_k(c, nt / (3 * (int64_t)S));
    double ts;
    if ((rc = time_per_gen(c, tier, b, ks, model, &ts)) != PT_OK) return rc;
    if (ts > cg) Rs = cta_samples(nt, ks) * np / (ts - cg);
  }
  c->tune_rate = R;
  c->tune_rate_stream = Rs;
  c->tune_fixed_s = cg;
  c->tune_model = model;
  c->tuned = true;
  return PT_OK;
}

double block_seconds(const pt_ctx* c, int tier, const HostDeBlock& b, int k) {
  const double R = resident(c, b.blk.ntiles, k) ? c->tune_rate : c->tune_rate_stream;
  const double per_gen = cta_samples(b.blk.ntiles, k) * npad_of(tier, b.pop) / R + c->tune_fixed_s;
  return per_gen * (b.gens + 1);
}

// Longest-processing-time assignment of blocks to `ng` groups; returns makespan.
double lpt(const std::vector<double>& t, int ng, std::vector<int>* sched, std::vector<int>* off) {
  std::vector<int> order(t.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return t[a] > t[b]; });
  typedef std::pair<double, int> Load;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int g = 0; g < ng; ++g) pq.push({0.0, g});
  std::vector<std::vector<int>> lists(ng);
  for (int i : order) {
    Load l = pq.top();
    pq.pop();
    lists[l.second].push_back(i);
    pq.push({l.first + t[i], l.second});
  }
  double makespan = 0.0;
  while (!pq.empty()) {
    makespan = std::max(makespan, pq.top().first);
    pq.pop();
  }
  if (sched && off) {
    sched->clear();
    off->assign(1, 0);
    for (auto& l : lists) {
      sched->insert(sched->end(), l.begin(), l.end());
      off->push_back((int)sched->size());
    }
  }
  return makespan;
}

void release(pt_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* bufs[] = {b->d_arena, b->d_amax, b->d_out, b->d_desc, b->d_ring, b->d_err};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  delete b;
}

// Block i's (lo, hi) pairs: the spec's five, then for the full model its
// two rows of ext_bounds (A1, f3).
void block_bounds(const pt_block_spec& s, const double* ext, int i, int dim, double* b) {
  std::memcpy(b, s.bounds, sizeof(double) * 10);
  if (dim == 7) std::memcpy(b + 10, ext + 4 * (size_t)i, sizeof(double) * 4);
}

int create_batch(pt_ctx* c, const pt_block_spec* specs, const double* ext_bounds, int nblocks, int tier,
                 int group_ctas, int model, pt_batch** out) {
  if (!c) return PT_EINVAL;
  const int dim = model == HOST_MODEL_FULL ? HOST_DMAX : HOST_D;
  if (!out || !specs || nblocks < 1 || !valid_tier(tier) || group_ctas < 0 || (dim == 7 && !ext_bounds))
    return fail(c, PT_EINVAL, "pt_batch_create: invalid argument");
  *out = nullptr;
  PT_CUDA(c, cudaSetDevice(c->device));
  int rc;
  for (int i = 0; i < nblocks; ++i) {
    const pt_block_spec& s = specs[i];
    double bnd[14];
    block_bounds(s, ext_bounds, i, dim, bnd);
    if ((rc = check_de_args(c, bnd, s.pop, s.gens, s.F, s.CR, tier, dim)) != PT_OK) return rc;
    if (!s.samples || s.n < 1 || esize_of(s.dtype) == 0 || !(s.scale > 0.0) || !(s.fs > 0.0) ||
        !std::isfinite(s.t0) || !std::isfinite(s.scale) || !std::isfinite(s.fs))
      return fail(c, PT_EINVAL, "pt_batch_create: invalid block " + std::to_string(i));
  }
  pt_batch* b = new (std::nothrow) pt_batch();
  if (!b) return PT_ENOMEM;
  b->ctx = c;
  b->tier = tier;
  b->model = model;
  b->dim = dim;
  b->nblocks = nblocks;
  auto bail = [&](int code) {
    release(b);
    return code;
  };
  // one arena for every block's samples, each padded with zeros to whole tiles
  std::vector<int64_t> offs(nblocks);
  int64_t total = 0;
  for (int i = 0; i < nblocks; ++i) {
    offs[i] = total;
    total += (padded_bytes(specs[i].n, esize_of(specs[i].dtype)) + 255) / 256 * 256;
  }
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_arena, total)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_amax, nblocks * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_out, (size_t)nblocks * (dim + 1) * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess || (e = cudaEventCreate(&b->ev0)) != cudaSuccess ||
      (e = cudaEventCreate(&b->ev1)) != cudaSuccess) {
    fail(c, e == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA,
         std::string("pt_batch_create: ") + cudaGetErrorString(e));
    return bail(e == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA);
  }
  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(b->d_arena, 0, total, s) != cudaSuccess ||
      cudaMemsetAsync(b->d_amax, 0, nblocks * sizeof(unsigned long long), s) != cudaSuccess)
    return bail(fail(c, PT_ECUDA, "pt_batch_create: memset failed"));
  for (int i = 0; i < nblocks; ++i) {
    const pt_block_spec& sp = specs[i];
    char* dst = (char*)b->d_arena + offs[i];
    if (cudaMemcpyAsync(dst, sp.samples, (size_t)sp.n * esize_of(sp.dtype), cudaMemcpyDefault, s) != cudaSuccess)
      return bail(fail(c, PT_ECUDA, "pt_batch_create: sample copy failed"));
    if ((rc = launch_absmax(c, s, dst, sp.n, sp.dtype, b->d_amax + i)) != PT_OK) return bail(rc);
  }
  std::vector<unsigned long long> amax(nblocks);
  if (cudaMemcpyAsync(amax.data(), b->d_amax, nblocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return bail(fail(c, PT_ECUDA, "pt_batch_create: absmax failed"));
  b->blocks.resize(nblocks);
  for (int i = 0; i < nblocks; ++i) {
    const pt_block_spec& sp = specs[i];
    HostDeBlock& h = b->blocks[i];
    double a;
    std::memcpy(&a, &amax[i], sizeof(a));
    h.blk.samples = (char*)b->d_arena + offs[i];
    h.blk.n = sp.n;
    h.blk.ntiles = (sp.n + HOST_L - 1) / HOST_L;
    h.blk.dtype = sp.dtype;
    h.blk.esize = esize_of(sp.dtype);
    h.blk.scale = sp.scale;
    h.blk.smax = a * sp.scale;
    h.blk.t0 = sp.t0;
    h.blk.fs = sp.fs;
    double bnd[14];
    block_bounds(sp, ext_bounds, i, dim, bnd);
    for (int j = 0; j < dim; ++j) {
      h.lo[j] = bnd[2 * j];
      h.hi[j] = bnd[2 * j + 1];
    }
    h.pop = sp.pop;
    h.gens = sp.gens;
    h.F = sp.F;
    h.CR = sp.CR;
    h.seed = sp.seed;
    h.block_id = sp.block_id;
    h.out = b->d_out + (size_t)i * (dim + 1);
    b->sample_evals += (double)sp.n * sp.pop * (sp.gens + 1);
  }
  // launch shape
  if ((rc = calibrate(c, tier, b->blocks[0], model)) != PT_OK) return bail(rc);
  std::vector<int> ks;
  if (group_ctas > 0) ks.push_back(clamp_k(c, group_ctas));
  else
    for (int k : {1, 2, 4, 8, 16, 37, 74, 148})
      if (k <= c->sms) ks.push_back(k);
  double best = 1e300;
  for (int k : ks) {
    std::vector<double> t(nblocks);
    for (int i = 0; i < nblocks; ++i) t[i] = block_seconds(c, tier, b->blocks[i], k);
    const int ng = std::min(c->sms / k, nblocks);
    const double m = lpt(t, ng, nullptr, nullptr);
    if (m < best) {
      best = m;
      b->k = k;
      b->ngroups = ng;
    }
  }
  {
    std::vector<double> t(nblocks);
    for (int i = 0; i < nblocks; ++i) t[i] = block_seconds(c, tier, b->blocks[i], b->k);
    lpt(t, b->ngroups, &b->sched, &b->off);
  }
  b->predicted_ms = best * 1e3;
  if ((e = cudaMalloc(&b->d_desc, de_desc_bytes(nblocks, b->ngroups))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_ring, (size_t)b->ngroups * RING_GROUP_WORDS * sizeof(unsigned long long))) !=
          cudaSuccess)
    return bail(fail(c, PT_ENOMEM, "pt_batch_create: descriptor allocation failed"));
  if ((rc = launch_de_groups(c, s, tier, b->blocks.data(), nblocks, b->sched.data(), b->off.data(), b->ngroups,
                             b->k, b->d_desc, b->d_ring, b->d_err, DE_UPLOAD, model)) != PT_OK)
    return bail(rc);
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(c, PT_ECUDA, "pt_batch_create: upload failed"));
  // capture the launch (ring/error clears + cooperative kernel) as a graph;
  // if the driver refuses, pt_batch_run launches directly
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int lr = launch_de_groups(c, cs, tier, b->blocks.data(), nblocks, b->sched.data(), b->off.data(),
                                      b->ngroups, b->k, b->d_desc, b->d_ring, b->d_err, DE_LAUNCH, model);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &g);
      ok = lr == PT_OK && ee == cudaSuccess && g != nullptr;
      if (ok && cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
        b->graph = g;
      } else {
        if (g) cudaGraphDestroy(g);
        b->exec = nullptr;
      }
    }
    cudaGetLastError();
    cudaStreamDestroy(cs);
    c->err.clear();
  }
  *out = b;
  return PT_OK;
}

}  // namespace

extern "C" {

int pt_batch_create(pt_ctx* c, const pt_block_spec* specs, int nblocks, int tier, int group_ctas, pt_batch** out) {
  return create_batch(c, specs, nullptr, nblocks, tier, group_ctas, HOST_MODEL_CUBIC, out);
}

int pt_batch_create_full(pt_ctx* c, const pt_block_spec* specs, const double* ext_bounds, int nblocks, int tier,
                         int group_ctas, pt_batch** out) {
  if (!c) return PT_EINVAL;
  if (c->objective != PT_OBJ_CHI2) return fail(c, PT_EINVAL, "the full model runs on the chi-square only");
  return create_batch(c, specs, ext_bounds, nblocks, tier, group_ctas, HOST_MODEL_FULL, out);
}

int pt_batch_run(pt_batch* b) {
  if (!b) return PT_EINVAL;
  pt_ctx* c = b->ctx;
  PT_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  PT_CUDA(c, cudaEventRecord(b->ev0, s));
  if (b->exec) {
    PT_CUDA(c, cudaGraphLaunch(b->exec, s));
  } else {
    const int rc = launch_de_groups(c, s, b->tier, b->blocks.data(), b->nblocks, b->sched.data(), b->off.data(),
                                    b->ngroups, b->k, b->d_desc, b->d_ring, b->d_err, DE_LAUNCH, b->model);
    if (rc != PT_OK) return rc;
  }
  PT_CUDA(c, cudaEventRecord(b->ev1, s));
  const int rc = kernel_status(c, s, b->d_err);
  if (rc != PT_OK) return rc;
  PT_CUDA(c, cudaEventElapsedTime(&b->last_ms, b->ev0, b->ev1));
  return PT_OK;
}

int pt_batch_results_full(pt_batch* b, double* out) {
  if (!b || !out) return PT_EINVAL;
  pt_ctx* c = b->ctx;
  const int w = b->dim + 1;
  std::vector<double> h((size_t)b->nblocks * w);
  PT_CUDA(c, cudaMemcpyAsync(h.data(), b->d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < b->nblocks; ++i) {
    double* o = out + (size_t)i * 8;
    for (int j = 0; j < 7; ++j) o[j] = j < b->dim ? h[(size_t)i * w + j] : 0.0;
    o[7] = h[(size_t)i * w + b->dim];
  }
  return PT_OK;
}

int pt_batch_results(pt_batch* b, pt_fit* out) {
  if (!b || !out) return PT_EINVAL;
  std::vector<double> h((size_t)b->nblocks * 8);
  const int rc = pt_batch_results_full(b, h.data());
  if (rc != PT_OK) return rc;
  for (int i = 0; i < b->nblocks; ++i) {
    for (int j = 0; j < 5; ++j) out[i].params[j] = h[(size_t)i * 8 + j];
    out[i].sse = h[(size_t)i * 8 + 7];
  }
  return PT_OK;
}

int pt_batch_get_info(const pt_batch* b, pt_batch_info* info) {
  if (!b || !info) return PT_EINVAL;
  info->nblocks = b->nblocks;
  info->ngroups = b->ngroups;
  info->group_ctas = b->k;
  info->tier = b->tier;
  info->uses_graph = b->exec ? 1 : 0;
  info->sample_evals = b->sample_evals;
  info->predicted_ms = b->predicted_ms;
  info->last_ms = b->last_ms;
  info->tune_rate = b->ctx->tune_rate;
  info->tune_gen_us = b->ctx->tune_fixed_s * 1e6;
  info->tune_rate_stream = b->ctx->tune_rate_stream;
  return PT_OK;
}

void pt_batch_destroy(pt_batch* b) {
  if (!b) return;
  cudaSetDevice(b->ctx->device);
  cudaStreamSynchronize(b->ctx->stream);
  release(b);
}

}  // extern "C"
