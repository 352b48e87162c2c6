// Serving loop of libphasetrack (pt_submit / pt_poll) and the block-to-block
// tracking helpers (pt_warm_bounds, pt_continuity).
//
// A worker thread per context owns a fixed number of device slots. Each slot
// has its own CUDA stream, sample buffer, DE ring, error word and pinned
// result buffer. The worker repeatedly (1) retires slots whose completion
// event has fired, turning them into results, and (2) admits queued blocks
// into free slots while the slots' sample buffers stay within the device
// memory budget. An admitted block is copied to its slot, its max |sample|
// is measured, and its DE runs as a cooperative launch of a few CTAs on the
// slot's stream, so blocks that arrive while others run overlap on the
// device. The GPU work is the same kernel and the same arithmetic as
// pt_de_solve_ex, so each fit is bit-identical to solving the block alone.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pt_internal.h"

using namespace pt;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Pending {
  uint64_t ticket;
  pt_request req;
  std::vector<unsigned char> samples;  // the caller's samples, copied at submit
  double t_submit;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* d_samples = nullptr;
  size_t cap = 0;
  unsigned long long* d_u64 = nullptr;
  unsigned long long* d_ring = nullptr;
  int* d_err = nullptr;
  double* d_out = nullptr;
  void* d_desc = nullptr;
  double* h_out = nullptr;  // pinned: 8 doubles (the fit, dim + 1 used) + the error word
  int dim = HOST_D;         // parameters of the running fit
  bool busy = false;
  uint64_t ticket = 0;
  int stream_id = 0;
  double t_submit = 0.0, t_admit = 0.0;
};

}  // namespace

struct pt_serve_state {
  pt_ctx wctx;  // the worker's own copy of the launch parameters and error text
  int max_inflight = 4, ctas = 0, max_queued = 64;
  size_t budget = 0, held = 0;
  std::vector<Slot> slots;
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, pt_result> done;
  std::unordered_map<uint64_t, int> live;  // queued or running tickets
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false, started = false;
};

namespace {

int slot_init(pt_serve_state* S, Slot& sl) {
  pt_ctx* w = &S->wctx;
  PT_CUDA(w, cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
  PT_CUDA(w, cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  PT_CUDA(w, cudaMalloc(&sl.d_u64, sizeof(unsigned long long)));
  PT_CUDA(w, cudaMalloc(&sl.d_ring, RING_GROUP_WORDS * sizeof(unsigned long long)));
  PT_CUDA(w, cudaMalloc(&sl.d_err, sizeof(int)));
  PT_CUDA(w, cudaMalloc(&sl.d_out, 8 * sizeof(double)));
  PT_CUDA(w, cudaMalloc(&sl.d_desc, de_desc_bytes(1, 1)));
  PT_CUDA(w, cudaMallocHost(&sl.h_out, 10 * sizeof(double)));
  return PT_OK;
}

void slot_free(Slot& sl) {
  if (sl.stream) cudaStreamSynchronize(sl.stream);
  void* d[] = {sl.d_samples, sl.d_u64, sl.d_ring, sl.d_err, sl.d_out, sl.d_desc};
  for (void* p : d)
    if (p) cudaFree(p);
  if (sl.h_out) cudaFreeHost(sl.h_out);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  sl = Slot();
}

size_t padded_bytes(const pt_block_spec& b) {
  return (size_t)((b.n + HOST_L - 1) / HOST_L * HOST_L) * esize_of(b.dtype);
}

// Start one block on a free slot (worker thread, lock held).
int admit(pt_serve_state* S, Slot& sl, Pending& p) {
  pt_ctx* w = &S->wctx;
  const pt_block_spec& b = p.req.block;
  const size_t need = padded_bytes(b);
  if (sl.cap < need) {
    if (sl.d_samples) cudaFree(sl.d_samples);
    S->held -= sl.cap;
    sl.d_samples = nullptr;
    sl.cap = 0;
  }
  const size_t before = sl.cap;
  HostDeBlock h;
  int rc = load_samples(w, sl.stream, p.samples.data(), b.n, b.dtype, b.scale, b.fs, b.t0, &sl.d_samples, &sl.cap,
                        sl.d_u64, &h.blk);
  S->held += sl.cap - before;
  if (rc != PT_OK) return rc;
  const bool full = p.req.model == PT_MODEL_FULL;
  const int dim = full ? HOST_DMAX : HOST_D;
  for (int j = 0; j < dim; ++j) {
    h.lo[j] = j < HOST_D ? b.bounds[2 * j] : p.req.ext_bounds[2 * (j - HOST_D)];
    h.hi[j] = j < HOST_D ? b.bounds[2 * j + 1] : p.req.ext_bounds[2 * (j - HOST_D) + 1];
  }
  h.pop = b.pop;
  h.gens = b.gens;
  h.F = b.F;
  h.CR = b.CR;
  h.seed = b.seed;
  h.block_id = b.block_id;
  h.out = sl.d_out;
  const int sched[1] = {0}, off[2] = {0, 1};
  const int k = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(h.blk.ntiles, S->ctas),
                                                             HOST_DE_GROUP_MAX));
  rc = launch_de_groups(w, sl.stream, p.req.tier, &h, 1, sched, off, 1, k, sl.d_desc, sl.d_ring, sl.d_err,
                        DE_UPLOAD | DE_LAUNCH, full ? HOST_MODEL_FULL : HOST_MODEL_CUBIC);
  if (rc != PT_OK) return rc;
  PT_CUDA(w, cudaMemcpyAsync(sl.h_out, sl.d_out, (dim + 1) * sizeof(double), cudaMemcpyDeviceToHost, sl.stream));
  PT_CUDA(w, cudaMemcpyAsync(sl.h_out + 8, sl.d_err, sizeof(int), cudaMemcpyDeviceToHost, sl.stream));
  sl.dim = dim;
  PT_CUDA(w, cudaEventRecord(sl.done, sl.stream));
  sl.busy = true;
  sl.ticket = p.ticket;
  sl.stream_id = p.req.stream_id;
  sl.t_submit = p.t_submit;
  sl.t_admit = now_s();
  return PT_OK;
}

void finish(pt_serve_state* S, uint64_t ticket, int stream_id, double t_submit, double t_admit, const double* out,
            int dim, int status) {
  pt_result r;
  std::memset(&r, 0, sizeof(r));
  if (out) {
    for (int j = 0; j < 5; ++j) r.fit.params[j] = out[j];
    if (dim == HOST_DMAX) {
      r.ext_params[0] = out[5];
      r.ext_params[1] = out[6];
    }
  }
  r.fit.sse = out ? out[dim] : 0.0;
  r.status = status;
  r.stream_id = stream_id;
  r.t_submit = t_submit;
  r.t_admit = t_admit;
  r.t_done = now_s();
  S->done[ticket] = r;
  S->live.erase(ticket);
}

void worker_loop(pt_serve_state* S) {
  cudaSetDevice(S->wctx.device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progressed = false;
    // retire finished slots
    for (Slot& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      int status = PT_OK;
      if (q != cudaSuccess) {
        cudaGetLastError();
        status = PT_ECUDA;
      } else {
        int derr;
        std::memcpy(&derr, sl.h_out + 8, sizeof(int));
        if (derr == 1) status = PT_ETIMEOUT;
        else if (derr != 0) status = PT_ECUDA;
      }
      finish(S, sl.ticket, sl.stream_id, sl.t_submit, sl.t_admit, status == PT_OK ? sl.h_out : nullptr, sl.dim,
             status);
      sl.busy = false;
      progressed = true;
    }
    // admit queued blocks while slots and memory allow
    while (!S->queue.empty()) {
      Slot* free_slot = nullptr;
      for (Slot& sl : S->slots)
        if (!sl.busy) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      Pending& p = S->queue.front();
      const size_t need = padded_bytes(p.req.block);
      if (need > free_slot->cap && S->held - free_slot->cap + need > S->budget) {
        // give back idle slots' buffers before refusing
        for (Slot& sl : S->slots)
          if (!sl.busy && sl.d_samples && &sl != free_slot) {
            cudaFree(sl.d_samples);
            S->held -= sl.cap;
            sl.d_samples = nullptr;
            sl.cap = 0;
          }
        if (S->held - free_slot->cap + need > S->budget) break;  // wait for running blocks to finish
      }
      Pending job = std::move(p);
      S->queue.pop_front();
      const int rc = admit(S, *free_slot, job);
      if (rc != PT_OK) finish(S, job.ticket, job.req.stream_id, job.t_submit, now_s(), nullptr, HOST_D, rc);
      progressed = true;
    }
    if (!progressed) S->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

int ensure_started(pt_ctx* c) {
  if (!c->serve) {
    pt_serve_state* S = new (std::nothrow) pt_serve_state();
    if (!S) return PT_ENOMEM;
    c->serve = S;
  }
  pt_serve_state* S = c->serve;
  if (S->started) return PT_OK;
  S->wctx.device = c->device;
  S->wctx.sms = c->sms;
  S->wctx.smem_optin = c->smem_optin;
  S->wctx.timeout_ns = c->timeout_ns;
  // the objective and strategy in force when the loop starts
  S->wctx.objective = c->objective;
  S->wctx.strategy = c->strategy;
  if (S->ctas <= 0) S->ctas = std::max(1, c->sms / S->max_inflight);
  if (S->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(c, PT_ECUDA, "serve: cudaMemGetInfo failed");
    S->budget = fr / 2;
  }
  S->slots.resize(S->max_inflight);
  for (Slot& sl : S->slots) {
    const int rc = slot_init(S, sl);
    if (rc != PT_OK) return fail(c, rc, S->wctx.err);
  }
  S->stop = false;
  S->worker = std::thread(worker_loop, S);
  S->started = true;
  return PT_OK;
}

}  // namespace

extern "C" {

double pt_clock(void) { return now_s(); }

void pt_serve_shutdown(pt_ctx* c) {
  if (!c || !c->serve) return;
  pt_serve_state* S = c->serve;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Slot& sl : S->slots) slot_free(sl);
  delete S;
  c->serve = nullptr;
}

int pt_serve_configure(pt_ctx* c, int max_inflight, int ctas_per_request, int64_t mem_budget_bytes,
                       int max_queued) {
  if (!c) return PT_EINVAL;
  if (max_inflight < 1 || max_inflight > 32 || ctas_per_request < 0 || mem_budget_bytes < 0 || max_queued < 1)
    return fail(c, PT_EINVAL, "pt_serve_configure: invalid argument");
  if (c->serve && c->serve->started) {
    std::lock_guard<std::mutex> lk(c->serve->mu);
    if (!c->serve->live.empty()) return fail(c, PT_EINVAL, "pt_serve_configure: requests in flight");
  }
  pt_serve_shutdown(c);
  pt_serve_state* S = new (std::nothrow) pt_serve_state();
  if (!S) return PT_ENOMEM;
  S->max_inflight = max_inflight;
  S->ctas = ctas_per_request;
  S->budget = (size_t)mem_budget_bytes;
  S->max_queued = max_queued;
  c->serve = S;
  return PT_OK;
}

int pt_submit(pt_ctx* c, const pt_request* req, uint64_t* ticket) {
  if (!c) return PT_EINVAL;
  if (!req || !ticket) return fail(c, PT_EINVAL, "pt_submit: invalid argument");
  const pt_block_spec& b = req->block;
  if (req->model != PT_MODEL_CUBIC && req->model != PT_MODEL_FULL)
    return fail(c, PT_EINVAL, "pt_submit: unknown model");
  const bool full = req->model == PT_MODEL_FULL;
  double bnd[14];
  std::memcpy(bnd, b.bounds, sizeof(double) * 10);
  if (full) std::memcpy(bnd + 10, req->ext_bounds, sizeof(double) * 4);
  int rc = check_de_args(c, bnd, b.pop, b.gens, b.F, b.CR, req->tier, full ? HOST_DMAX : HOST_D);
  if (rc != PT_OK) return rc;
  const int obj = c->serve && c->serve->started ? c->serve->wctx.objective : c->objective;
  if (full && obj != PT_OBJ_CHI2) return fail(c, PT_EINVAL, "pt_submit: the full model runs on the chi-square only");
  const int es = esize_of(b.dtype);
  if (!b.samples || b.n < 1 || es == 0 || !(b.scale > 0.0) || !(b.fs > 0.0) || !std::isfinite(b.t0) ||
      b.n > ((int64_t)1 << 36))
    return fail(c, PT_EINVAL, "pt_submit: invalid block");
  if ((rc = ensure_started(c)) != PT_OK) return rc;
  pt_serve_state* S = c->serve;
  if (padded_bytes(b) > S->budget) return fail(c, PT_EINVAL, "pt_submit: block larger than the memory budget");
  Pending p;
  p.req = *req;
  p.samples.resize((size_t)b.n * es);
  if (is_device_ptr(b.samples)) {
    PT_CUDA(c, cudaMemcpy(p.samples.data(), b.samples, p.samples.size(), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(p.samples.data(), b.samples, p.samples.size());
  }
  p.req.block.samples = nullptr;
  p.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->max_queued) return fail(c, PT_EAGAIN, "pt_submit: queue full");
    p.ticket = S->next_ticket++;
    *ticket = p.ticket;
    S->live[p.ticket] = 1;
    S->queue.push_back(std::move(p));
  }
  S->cv.notify_all();
  return PT_OK;
}

int pt_poll(pt_ctx* c, uint64_t ticket, pt_result* out) {
  if (!c || !out) return PT_EINVAL;
  if (!c->serve) return fail(c, PT_EINVAL, "pt_poll: unknown ticket");
  pt_serve_state* S = c->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it != S->done.end()) {
    *out = it->second;
    S->done.erase(it);
    return PT_OK;
  }
  if (S->live.count(ticket)) return PT_PENDING;
  return fail(c, PT_EINVAL, "pt_poll: unknown ticket");
}

// ---- tracking helpers (Sec. 3.1.1 running-time ranges, Eq. 3-1-2) ----------

int pt_warm_bounds(const double prev[5], double dt, double T_next, double min_f0, double min_f1, double min_f2,
                   double bounds_out[10]) {
  if (!prev || !bounds_out || !(T_next > 0.0) || !std::isfinite(dt)) return PT_EINVAL;
  for (int j = 0; j < 5; ++j)
    if (!std::isfinite(prev[j])) return PT_EINVAL;
  if (!(min_f0 > 0.0)) min_f0 = 2.0 / T_next;
  if (!(min_f1 > 0.0)) min_f1 = 4.0 / (T_next * T_next);
  if (!(min_f2 > 0.0)) min_f2 = 24.0 / (T_next * T_next * T_next);
  const double A = prev[0], f0 = prev[2], f1 = prev[3], f2 = prev[4];
  // frequency (Hz, Eq. 3-1-1 in cycles) and its rate, extrapolated from block n
  auto freq = [&](double t) { return f0 + f1 * t + f2 * t * t / 2.0; };
  auto rate = [&](double t) { return f1 + f2 * t; };
  // the span of block n+1: from its left border to its right border
  const double ta = dt - T_next / 2.0, tb = dt + T_next / 2.0;
  const double fc = freq(dt), rc = rate(dt);
  double flo = std::min(std::min(freq(ta), freq(tb)), fc), fhi = std::max(std::max(freq(ta), freq(tb)), fc);
  double rlo = std::min(rate(ta), rate(tb)), rhi = std::max(rate(ta), rate(tb));
  // ranges are about block n+1's centre values: keep them covering fc, rc
  bounds_out[0] = std::fabs(A) * 0.9;
  bounds_out[1] = std::fabs(A) * 1.1;
  bounds_out[2] = -3.14159265358979323846;
  bounds_out[3] = 3.14159265358979323846;
  bounds_out[4] = std::min(flo, fc - min_f0);
  bounds_out[5] = std::max(fhi, fc + min_f0);
  bounds_out[6] = std::min(rlo, rc - min_f1);
  bounds_out[7] = std::max(rhi, rc + min_f1);
  bounds_out[8] = f2 - min_f2;
  bounds_out[9] = f2 + min_f2;
  return PT_OK;
}

int pt_warm_bounds_full(const double prev[7], double dt, double T_next, const double a1_range[2],
                        double bounds_out[14]) {
  if (!prev || !bounds_out || !(T_next > 0.0) || !std::isfinite(dt)) return PT_EINVAL;
  for (int j = 0; j < 7; ++j)
    if (!std::isfinite(prev[j])) return PT_EINVAL;
  if (a1_range && (!std::isfinite(a1_range[0]) || !std::isfinite(a1_range[1]) || a1_range[0] > a1_range[1]))
    return PT_EINVAL;
  const double T = T_next;
  const double min_f0 = 2.0 / T, min_f1 = 4.0 / (T * T), min_f2 = 24.0 / (T * T * T),
               min_f3 = 192.0 / (T * T * T * T);
  const double A = prev[0], f0 = prev[2], f1 = prev[3], f2 = prev[4], A1 = prev[5], f3 = prev[6];
  // frequency (Hz), its rate and the rate's derivative of the quartic phase, extrapolated from block n
  auto freq = [&](double t) { return f0 + f1 * t + f2 * t * t / 2.0 + f3 * t * t * t / 6.0; };
  auto rate = [&](double t) { return f1 + f2 * t + f3 * t * t / 2.0; };
  auto jerk = [&](double t) { return f2 + f3 * t; };
  const double ta = dt - T / 2.0, tb = dt + T / 2.0;
  auto span = [&](auto fn, double mw, double* lo, double* hi) {
    const double c = fn(dt);
    *lo = std::min(std::min(std::min(fn(ta), fn(tb)), c), c - mw);
    *hi = std::max(std::max(std::max(fn(ta), fn(tb)), c), c + mw);
  };
  const double An = std::fabs(A + A1 * dt);  // the amplitude at block n+1's centre
  bounds_out[0] = An * 0.9;
  bounds_out[1] = An * 1.1;
  bounds_out[2] = -3.14159265358979323846;
  bounds_out[3] = 3.14159265358979323846;
  span(freq, min_f0, &bounds_out[4], &bounds_out[5]);
  span(rate, min_f1, &bounds_out[6], &bounds_out[7]);
  span(jerk, min_f2, &bounds_out[8], &bounds_out[9]);
  if (a1_range) {
    bounds_out[10] = a1_range[0];
    bounds_out[11] = a1_range[1];
  } else {
    bounds_out[10] = A1 - 0.2 * An / T;
    bounds_out[11] = A1 + 0.2 * An / T;
  }
  bounds_out[12] = f3 - min_f3;
  bounds_out[13] = f3 + min_f3;
  return PT_OK;
}

int pt_continuity_full(const double a[7], double Ta, const double b[7], double Tb, double max_dphi,
                       double max_dfreq, double* dphi, double* dfreq) {
  if (!a || !b || !dphi || !dfreq || !(Ta > 0.0) || !(Tb > 0.0)) return PT_EINVAL;
  const double TWO_PI = 2.0 * 3.14159265358979323846;
  // Eq. 3-1-1 carried to order 4: phase (rad) and frequency (rad/s)
  auto phase = [&](const double* th, double t) {
    return th[1] + TWO_PI * (th[2] * t + th[3] * t * t / 2.0 + th[4] * t * t * t / 6.0 +
                             th[6] * t * t * t * t / 24.0);
  };
  auto freq = [&](const double* th, double t) {
    return TWO_PI * (th[2] + th[3] * t + th[4] * t * t / 2.0 + th[6] * t * t * t / 6.0);
  };
  double d = std::fmod(phase(a, Ta / 2.0) - phase(b, -Tb / 2.0), TWO_PI);
  if (d > TWO_PI / 2.0) d -= TWO_PI;
  if (d < -TWO_PI / 2.0) d += TWO_PI;
  *dphi = std::fabs(d);
  *dfreq = std::fabs(freq(a, Ta / 2.0) - freq(b, -Tb / 2.0));
  return (*dphi <= max_dphi && *dfreq <= max_dfreq) ? 1 : 0;
}

int pt_continuity(const double a[5], double Ta, const double b[5], double Tb, double max_dphi, double max_dfreq,
                  double* dphi, double* dfreq) {
  if (!a || !b || !dphi || !dfreq || !(Ta > 0.0) || !(Tb > 0.0)) return PT_EINVAL;
  const double PI = 3.14159265358979323846;
  // Eq. 3-1-1 in the paper's coefficients: c0 = phi0, c1 = 2 pi f0, c2 = pi f1, c3 = pi f2 / 3
  auto phase = [&](const double* th, double t) {
    return th[1] + 2.0 * PI * th[2] * t + PI * th[3] * t * t + PI * th[4] / 3.0 * t * t * t;
  };
  auto freq = [&](const double* th, double t) {
    return 2.0 * PI * th[2] + 2.0 * PI * th[3] * t + PI * th[4] * t * t;
  };
  double d = std::fmod(phase(a, Ta / 2.0) - phase(b, -Tb / 2.0), 2.0 * PI);
  if (d > PI) d -= 2.0 * PI;
  if (d < -PI) d += 2.0 * PI;
  *dphi = std::fabs(d);
  *dfreq = std::fabs(freq(a, Ta / 2.0) - freq(b, -Tb / 2.0));
  return (*dphi <= max_dphi && *dfreq <= max_dfreq) ? 1 : 0;
}

}  // extern "C"
