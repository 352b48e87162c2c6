// Block-to-block tracking of one station stream (pt_track_*): the data
// process flow of Sec. 3.1.4 around the DE fit of each block. Running-time
// ranges (Sec. 3.1.1), the continuity check of Eq. 3-1-2, range enlargement
// and retry with abandonment after max_attempts searches, and the total-phase
// / integration-Doppler chaining of Eq. 4-1-2. Host code only: every fit is
// pt_de_solve_ex (cubic model) or pt_de_solve_full (the full model: amplitude
// slope and order-4 phase, Sec. 3.2) on the session's context.
#include <cmath>
#include <cstring>
#include <limits>
#include <new>

#include "pt_internal.h"

using namespace pt;

namespace {

constexpr double TWO_PI_D = 6.283185307179586476925286766559;
const double NaN = std::numeric_limits<double>::quiet_NaN();

// Phase (rad, not reduced) and frequency (rad/s) at t from the block centre
// (Eq. 3-1-1 in cycles form) of p = (A, phi0, f0, f1, f2, A1, f3); f3 = 0 for
// the cubic model.
double phase_at(const double* p, double t) {
  return p[1] + TWO_PI_D * (p[2] * t + p[3] * t * t / 2.0 + p[4] * t * t * t / 6.0 + p[6] * t * t * t * t / 24.0);
}
double freq_at(const double* p, double t) {
  return TWO_PI_D * (p[2] + p[3] * t + p[4] * t * t / 2.0 + p[6] * t * t * t / 6.0);
}
double wrap_2pi(double x) {
  double r = std::fmod(x, TWO_PI_D);
  return r < 0.0 ? r + TWO_PI_D : r;
}

// Finite (lo, hi) pairs with lo <= hi (lo == hi holds the parameter fixed).
bool finite_bounds(const double* b, int dim) {
  for (int j = 0; j < dim; ++j)
    if (!std::isfinite(b[2 * j]) || !std::isfinite(b[2 * j + 1]) || !(b[2 * j] <= b[2 * j + 1])) return false;
  return true;
}

// A parameter whose initial range is a point stays there in every search
// (e.g. f3 = 0 for the paper's 6-parameter model, or the constant amplitude
// of the correlation objective, Eq. 2-2-6).
void keep_fixed(double* b, const double* init, int dim) {
  for (int j = 0; j < dim; ++j)
    if (init[2 * j] == init[2 * j + 1]) b[2 * j] = b[2 * j + 1] = init[2 * j];
}

// Widen the f0, f1, f2 and A ranges (and the full model's f3) about their
// centres by `e` (phi0 keeps its range, A1 its session range); A stays positive.
void enlarge_bounds(double* b, double e, int dim) {
  for (int j : {0, 2, 3, 4, 6}) {
    if (j >= dim) break;
    const double c = 0.5 * (b[2 * j] + b[2 * j + 1]), h = 0.5 * (b[2 * j + 1] - b[2 * j]) * e;
    b[2 * j] = c - h;
    b[2 * j + 1] = c + h;
  }
  if (b[0] <= 0.0 && b[1] > 0.0) b[0] = 1e-3 * b[1];
}

}  // namespace

struct pt_track {
  pt_ctx* ctx = nullptr;
  pt_track_config cfg{};
  int dim = 5;             // 5: the cubic model, 7: the full model
  double init[14] = {};
  int64_t next_index = 0;
  bool have_ref = false;   // an accepted fit exists
  bool adjacent = false;   // the previous block was accepted (continuity applies)
  double ref[7] = {};      // the last accepted fit (A1 = f3 = 0 for the cubic model)
  double ref_T = 0.0;      // its block length
  double ref_to_end = 0.0; // time from its centre to the end of the last block processed
  double acc_phase = 0.0, acc_T = 0.0;  // current count interval (Eq. 4-1-2)
};

namespace {

int create_session(pt_ctx* ctx, const pt_track_config* cfg, const double* bounds, int dim, pt_track** out) {
  if (!ctx || !cfg || !bounds || !out) return PT_EINVAL;
  *out = nullptr;
  if (cfg->pop < 4 || cfg->pop > PT_POP_MAX || cfg->gens < 0 || !(cfg->F > 0.0) || !std::isfinite(cfg->F) ||
      !(cfg->CR >= 0.0) || !std::isfinite(cfg->CR) || !valid_tier(cfg->tier) || !(cfg->max_dphi > 0.0) ||
      !(cfg->max_dfreq > 0.0) || !(cfg->enlarge >= 1.0) || !std::isfinite(cfg->enlarge) ||
      cfg->max_attempts < 1 || std::isnan(cfg->count_interval) || !finite_bounds(bounds, dim))
    return fail(ctx, PT_EINVAL, "pt_track_create: invalid configuration or bounds");
  pt_track* t = new (std::nothrow) pt_track;
  if (!t) return fail(ctx, PT_ENOMEM, "pt_track_create: out of host memory");
  t->ctx = ctx;
  t->cfg = *cfg;
  t->dim = dim;
  std::memcpy(t->init, bounds, sizeof(double) * 2 * dim);
  *out = t;
  return PT_OK;
}

}  // namespace

extern "C" {

int pt_track_create(pt_ctx* ctx, const pt_track_config* cfg, const double bounds[10], pt_track** out) {
  return create_session(ctx, cfg, bounds, 5, out);
}

int pt_track_create_full(pt_ctx* ctx, const pt_track_config* cfg, const double bounds[14], pt_track** out) {
  return create_session(ctx, cfg, bounds, 7, out);
}

void pt_track_destroy(pt_track* t) { delete t; }

int pt_track_block(pt_track* t, const void* samples, int64_t n, int dtype, double scale, double fs,
                   pt_track_result* out) {
  if (!t || !samples || !out || n < 1 || !(fs > 0.0) || !std::isfinite(fs)) return PT_EINVAL;
  const pt_track_config& c = t->cfg;
  const double T = (double)n / fs;
  int rc = pt_load_block(t->ctx, samples, n, dtype, scale, fs, -(double)(n - 1) / (2.0 * fs));
  if (rc != PT_OK) return rc;
  const bool full = t->dim == 7;
  double b[14];
  if (!t->have_ref) {
    std::memcpy(b, t->init, sizeof(double) * 2 * t->dim);
  } else if (full) {
    // the amplitude slope keeps the session's initial range (Sec. 3.1.1: the
    // range of c5 can be fixed)
    if ((rc = pt_warm_bounds_full(t->ref, t->ref_to_end + 0.5 * T, T, t->init + 10, b)) != PT_OK) return rc;
  } else if ((rc = pt_warm_bounds(t->ref, t->ref_to_end + 0.5 * T, T, 0.0, 0.0, 0.0, b)) != PT_OK) {
    return rc;
  }
  keep_fixed(b, t->init, t->dim);
  double p[8] = {};  // (A, phi0, f0, f1, f2, A1, f3) and the SSE; A1 = f3 = 0 for the cubic model
  double sse = 0.0;
  double dphi = NaN, dfreq = NaN;
  int quality = 0, attempts = 0;
  for (int a = 1; a <= c.max_attempts; ++a) {
    attempts = a;
    const uint64_t seed = c.seed + (uint64_t)(a - 1);
    if (full) {
      if ((rc = pt_de_solve_full(t->ctx, b, c.pop, c.gens, c.F, c.CR, seed, (uint32_t)t->next_index, p, nullptr,
                                 nullptr, c.tier)) != PT_OK)
        return rc;
      sse = p[7];
    } else {
      double q[6];
      if ((rc = pt_de_solve_ex(t->ctx, b, c.pop, c.gens, c.F, c.CR, seed, (uint32_t)t->next_index, q, nullptr,
                               nullptr, c.tier)) != PT_OK)
        return rc;
      std::memcpy(p, q, sizeof(double) * 5);
      sse = q[5];
    }
    if (!t->adjacent) {
      dphi = dfreq = NaN;
      quality = a;
      break;
    }
    const int ok = full ? pt_continuity_full(t->ref, t->ref_T, p, T, c.max_dphi, c.max_dfreq, &dphi, &dfreq)
                        : pt_continuity(t->ref, t->ref_T, p, T, c.max_dphi, c.max_dfreq, &dphi, &dfreq);
    if (ok < 0) return ok;
    if (ok == 1) {
      quality = a;
      break;
    }
    if (a < c.max_attempts) {
      enlarge_bounds(b, c.enlarge, t->dim);
      keep_fixed(b, t->init, t->dim);
    }
  }
  pt_track_result r{};
  r.block_index = t->next_index++;
  r.quality = quality;
  r.attempts = attempts;
  std::memcpy(r.params, p, sizeof(r.params));
  r.sse = sse;
  r.dphi = dphi;
  r.dfreq = dfreq;
  r.phi_left = wrap_2pi(phase_at(p, -0.5 * T));
  r.phi_right = wrap_2pi(phase_at(p, 0.5 * T));
  r.f_left = freq_at(p, -0.5 * T);
  r.f_right = freq_at(p, 0.5 * T);
  r.int_doppler = NaN;
  r.interval_phase = NaN;
  std::memcpy(r.bounds, b, sizeof(double) * 2 * t->dim);
  if (quality > 0) {
    // Eq. 4-1-2 term: the odd part of the phase across the block (the even
    // f1 and f3 terms cancel between the borders)
    r.total_phase = TWO_PI_D * (p[2] * T + p[4] * T * T * T / 24.0);
    std::memcpy(t->ref, p, sizeof(t->ref));
    t->ref_T = T;
    t->ref_to_end = 0.5 * T;
    t->have_ref = true;
    t->adjacent = true;
    if (c.count_interval > 0.0) {
      t->acc_phase += r.total_phase;
      t->acc_T += T;
      if (t->acc_T >= c.count_interval * (1.0 - 1e-12)) {
        r.interval_phase = t->acc_phase;
        r.int_doppler = t->acc_phase / t->acc_T;
        t->acc_phase = 0.0;
        t->acc_T = 0.0;
      }
    }
  } else {
    // abandoned: no adjacent reference for the next block, the count interval is broken
    r.total_phase = NaN;
    t->adjacent = false;
    if (t->have_ref) t->ref_to_end += T;
    t->acc_phase = 0.0;
    t->acc_T = 0.0;
  }
  *out = r;
  return PT_OK;
}

}  // extern "C"
