/*
 * Plain FP64 CPU oracle for the DE phase-tracking hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline / reference leg may load, call or execute this
 * code. The CUDA library shares no code with it: nothing here is included,
 * linked or generated for the GPU path, and nothing here reads the GPU path.
 *
 * What it computes (arxiv 1906.10598):
 *   - Signal model, Sec. 2.2 Eq. 2-2-2 with the amplitude slope c5 = 0 and
 *     the Taylor phase of Eq. 2-2-1 / Eq. 2-2-3, re-parameterised in cycles:
 *       m(t) = A cos(2 pi p(t)),  p(t) = phi0/(2 pi) + f0 t + f1 t^2/2 + f2 t^3/6
 *     i.e. c0 = phi0, c1 = 2 pi f0, c2 = pi f1, c3 = pi f2 / 3, c4 = A.
 *   - The full model: Eq. 2-2-2 with the amplitude slope c5 = A1 and the
 *     phase of Eq. 2-2-1 taken to order n = 4 (Sec. 3.2, for arcs near
 *     perigee), theta = (A, phi0, f0, f1, f2, A1, f3):
 *       m(t) = (A + A1 t) cos(2 pi p(t)),  p(t) = ... + f3 t^4 / 24,
 *     fitted on the chi-square by the same DE over 7 parameters.
 *   - Chi-square objective with unit weights, Sec. 2.2 Eq. 2-2-4:
 *       F(theta) = sum_i (s_i - m(t_i))^2.
 *   - Correlation objective, Sec. 2.2 Eq. 2-2-5 with the constant-amplitude
 *     model of Eq. 2-2-6:
 *       cor(theta) = sum_i s_i m(t_i),  F_cor(theta) = 1 / (atan(cor) + pi/2).
 *     "cor" is read as the unnormalised cross-correlation: the paper states
 *     F_cor converges to 1/pi, which a normalised coefficient (at most 1)
 *     cannot reach; A is held constant by the caller (the paper's "average
 *     amplitude"), since a fitted A makes F_cor divergent.
 *   - Differential Evolution, Sec. 1.2 (mutation -> crossover -> selection,
 *     Fig. "DE algorithm iteration flowchart") with the controls of Sec. 3.1.2
 *     Table 3-1-1 (F, CR, fixed itermax as the stop rule).  The mutation
 *     strategy is DE/rand/1 with binomial crossover by default; the paper
 *     names its strategies only by number, and its "3" and "6" are read as
 *     DE/best/1 with jitter and the DE/rand/1 either-or algorithm (see
 *     oc_de_run_strategy).
 *   - Derived observables: phase and instantaneous frequency, Sec. 3.1.3
 *     Eq. 3-1-1; block total-count phase, Sec. 4.1.1 Eq. 4-1-2.
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from
 *     the published definition.
 *
 * Readings where the paper is silent (each restated in the design notes):
 *   t_i = t0 + i/fs; SSE accumulated in long double in index order; the
 *   fractional cycle is p - nearbyint(p) before the 2 pi scaling; DE index
 *   draws use Lemire's multiply-shift on one 32-bit word with index shifting
 *   (no rejection); crossover compares a raw 32-bit word against
 *   floor(CR 2^32); out-of-range trial components are pulled to the midpoint
 *   of the violated bound and the parent's component, except phi0 whose range
 *   is the full circle, which wraps; selection keeps the trial on ties; the
 *   final answer is the lowest-index minimum.
 *
 * Parity pins live in the test suite (closed-form tone sums, noise-energy
 * identities, brute-force grids, cuRAND/Random123 known answers, textbook
 * DE test functions, the paper's Appendix 1 worked example; for the full
 * model, finite differences of the quartic phase and closed-form sums at
 * sixteenth-cycle sample phases).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_D 5
static const double OC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11): 10 rounds of a two-multiplier
 * Feistel-like bijection on a 128-bit counter, keyed by a 64-bit key that is
 * bumped by the Weyl constants between rounds. */
static const uint32_t PHILOX_MUL0 = 0xD2511F53u, PHILOX_MUL1 = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL0 = 0x9E3779B9u, PHILOX_WEYL1 = 0xBB67AE85u;

void oc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_WEYL0; k1 += PHILOX_WEYL1; }
    uint64_t p0 = (uint64_t)PHILOX_MUL0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_MUL1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Twelve words for DE draws of individual `ind` at generation `gen` of block
 * `block_id`: counters (group, ind, gen, block_id) for group = 0, 1, 2. */
static void oc_draw12(uint64_t seed, uint32_t block_id, uint32_t gen, uint32_t ind, uint32_t w[12]) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (uint32_t g = 0; g < 3; ++g) {
    uint32_t ctr[4] = {g, ind, gen, block_id};
    oc_philox4x32_10(ctr, key, w + 4 * g);
  }
}

/* Uniform double in [0,1) with 53 random bits (27 from a, 26 from b). */
static double oc_u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* Integer in [0, k) by Lemire's multiply-shift of one 32-bit word. */
static uint32_t oc_lemire(uint32_t w, uint32_t k) { return (uint32_t)(((uint64_t)w * k) >> 32); }

/* ------------------------------------------------------------------------ */
/* Model and objective (Eq. 2-2-1..2-2-4, c5 = 0). */

double oc_phase_cycles(const double th[OC_D], double t) {
  return th[1] / (2.0 * OC_PI) + th[2] * t + th[3] * t * t / 2.0 + th[4] * t * t * t / 6.0;
}

double oc_model(const double th[OC_D], double t) {
  double p = oc_phase_cycles(th, t);
  double r = p - nearbyint(p); /* fractional cycle in [-1/2, 1/2] */
  return th[0] * cos(2.0 * OC_PI * r);
}

double oc_sse(const double* s, int64_t n, double fs, double t0, const double th[OC_D]) {
  long double acc = 0.0L;
  for (int64_t i = 0; i < n; ++i) {
    double t = t0 + (double)i / fs;
    double res = s[i] - oc_model(th, t);
    acc += (long double)res * (long double)res;
  }
  return (double)acc;
}

/* The full model of Sec. 2.2: Eq. 2-2-2 with the amplitude slope (c5) and the
 * Taylor phase of Eq. 2-2-1 at order n = 4 (the paper's order for
 * high-dynamics arcs near perigee, Sec. 3.2), theta = (A, phi0, f0, f1, f2,
 * A1, f3):
 *   m(t) = (A + A1 t) cos(2 pi p(t)),
 *   p(t) = phi0/(2 pi) + f0 t + f1 t^2/2 + f2 t^3/6 + f3 t^4/24. */
#define OC_DF 7

double oc_phase_cycles_full(const double th[OC_DF], double t) {
  return th[1] / (2.0 * OC_PI) + th[2] * t + th[3] * t * t / 2.0 + th[4] * t * t * t / 6.0 +
         th[6] * t * t * t * t / 24.0;
}

double oc_model_full(const double th[OC_DF], double t) {
  double p = oc_phase_cycles_full(th, t);
  double r = p - nearbyint(p);
  return (th[0] + th[5] * t) * cos(2.0 * OC_PI * r);
}

double oc_sse_full(const double* s, int64_t n, double fs, double t0, const double th[OC_DF]) {
  long double acc = 0.0L;
  for (int64_t i = 0; i < n; ++i) {
    double t = t0 + (double)i / fs;
    double res = s[i] - oc_model_full(th, t);
    acc += (long double)res * (long double)res;
  }
  return (double)acc;
}

void oc_sse_full_many(const double* s, int64_t n, double fs, double t0, const double* cands, int64_t ncand,
                      double* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t c = 0; c < ncand; ++c) out[c] = oc_sse_full(s, n, fs, t0, cands + OC_DF * c);
}

/* Eq. 2-2-5 / 2-2-6: the unnormalised cross-correlation of the samples with
 * the model (long double, index order) and the correlation objective. */
double oc_cor(const double* s, int64_t n, double fs, double t0, const double th[OC_D]) {
  long double acc = 0.0L;
  for (int64_t i = 0; i < n; ++i) {
    double t = t0 + (double)i / fs;
    acc += (long double)s[i] * (long double)oc_model(th, t);
  }
  return (double)acc;
}

double oc_cor_objective(const double* s, int64_t n, double fs, double t0, const double th[OC_D]) {
  return 1.0 / (atan(oc_cor(s, n, fs, t0, th)) + OC_PI / 2.0);
}

void oc_cor_objective_many(const double* s, int64_t n, double fs, double t0, const double* cands, int64_t ncand,
                           double* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t c = 0; c < ncand; ++c) out[c] = oc_cor_objective(s, n, fs, t0, cands + OC_D * c);
}

/* SSE for `ncand` candidate rows (row-major, 5 per row). */
void oc_sse_many(const double* s, int64_t n, double fs, double t0, const double* cands, int64_t ncand,
                 double* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t c = 0; c < ncand; ++c) out[c] = oc_sse(s, n, fs, t0, cands + OC_D * c);
}

/* ------------------------------------------------------------------------ */
/* Differential Evolution, DE/rand/1/bin, synchronous generations.
 * The objective is a callback so that the same DE can be checked on textbook
 * functions; `oc_de_solve_block` binds it to the chi-square objective. */

typedef double (*oc_objective_fn)(const double* th, void* user);

/* The phi0 component (index 1) wraps when its range spans a full circle
 * (Sec. 3.1.1: the phase range is [0, 2 pi]). */
static int oc_is_periodic(int j, const double* lo, const double* hi) {
  return j == 1 && (hi[j] - lo[j]) >= 2.0 * OC_PI * (1.0 - 1e-12);
}

static double oc_repair(int j, double u, double parent, const double* lo, const double* hi) {
  if (oc_is_periodic(j, lo, hi)) {
    double two_pi = 2.0 * OC_PI;
    double k = floor((u - lo[j]) / two_pi);
    return u - k * two_pi;
  }
  if (u < lo[j]) return (lo[j] + parent) / 2.0;
  if (u > hi[j]) return (hi[j] + parent) / 2.0;
  return u;
}

/* Three distinct indices different from i, drawn without rejection: the
 * first from NP-1 slots, the second from NP-2, the third from NP-3, each
 * mapped onto the remaining indices in ascending order. Exported so the test
 * suite can feed it chosen words. */
void oc_pick3(uint32_t i, uint32_t np, const uint32_t w[3], uint32_t r[3]) {
  uint32_t excl[4];
  uint32_t nex = 1;
  excl[0] = i;
  for (int d = 0; d < 3; ++d) {
    uint32_t v = oc_lemire(w[d], np - 1 - (uint32_t)d);
    /* excl is kept sorted ascending */
    for (uint32_t e = 0; e < nex; ++e)
      if (v >= excl[e]) v++;
    r[d] = v;
    /* insert v into the sorted exclusion list */
    uint32_t pos = nex;
    while (pos > 0 && excl[pos - 1] > v) { excl[pos] = excl[pos - 1]; --pos; }
    excl[pos] = v;
    nex++;
  }
}

/* Mutation strategies. Table 3-1-1 names the strategy only by number
 * ("3 | 6": the third for the chi-square, the sixth for the correlation
 * objective, Sec. 3.1.2) and counts six, citing Price, Storn & Lampinen,
 * "Differential Evolution: A Practical Approach to Global Optimization"
 * (2006); the third and sixth are read in that book's order. With r1, r2,
 * r3 the three drawn indices (all different from i and each other):
 *   OC_DE_RAND1_BIN    v = x_r1 + F (x_r2 - x_r3), binomial crossover (the
 *                      textbook default, used when no strategy is named);
 *   OC_DE_BEST1_JITTER v_j = x_best,j + F_j (x_r2,j - x_r3,j) with the
 *                      per-component jitter F_j = F + 1e-4 U_j (U_j uniform
 *                      in [0,1)), binomial crossover; x_best is the
 *                      lowest-index minimum of the previous generation;
 *   OC_DE_EITHER_OR    with probability 1/2 the rand/1 mutant, otherwise the
 *                      three-point recombination v = x_r1 + K ((x_r2 + x_r3)
 *                      - 2 x_r1), K = (F + 1)/2; the trial is v itself (no
 *                      crossover). */
#define OC_DE_RAND1_BIN 0
#define OC_DE_BEST1_JITTER 3
#define OC_DE_EITHER_OR 6

/* Sixteen words (counter groups 0..3) for individual ind at generation gen;
 * the first twelve are oc_draw12's. */
static void oc_draw16(uint64_t seed, uint32_t block_id, uint32_t gen, uint32_t ind, uint32_t w[16]) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (uint32_t g = 0; g < 4; ++g) {
    uint32_t ctr[4] = {g, ind, gen, block_id};
    oc_philox4x32_10(ctr, key, w + 4 * g);
  }
}

/* The jitter and either-or words of individual ind at generation gen: words
 * 9..11 of the three-group draw, then a fourth counter group (word group 3). */
static void oc_draw_extra(uint64_t seed, uint32_t block_id, uint32_t gen, uint32_t ind, uint32_t w4[4]) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {3u, ind, gen, block_id};
  oc_philox4x32_10(ctr, key, w4);
}

int oc_de_run_dim(oc_objective_fn obj, void* user, int dim, const double* bounds, int np, int gens, double F,
                  double CR, uint64_t seed, uint32_t block_id, int strategy, double* out, double* final_pop,
                  double* final_fit, int nthreads);

/* The trials of generation g >= 1 (Sec. 1.2: mutation, then crossover), from
 * the population x (np x dim) of generation g-1 and its fitness fx, with the
 * bound repair. For each individual i: three indices r from oc_pick3 on
 * words 0..2 of its counter group draw, jrand = Lemire(word 3, dim), the
 * crossover mask (component j comes from the mutant when j = jrand, CR >= 1
 * or word 4+j < floor(CR 2^32)), the strategy's mutant, and the repair of
 * every component taken from the mutant. Optional outputs (NULL to skip):
 * r_out (np x 3), jrand_out (np), take_out (np, bit j = component j from the
 * mutant), three_point_out (np, the either-or strategy's coin), best_out (the
 * previous generation's lowest-index minimum, used by DE/best/1). */
static void oc_generation_trials(uint64_t seed, uint32_t block_id, uint32_t g, int np, int dim, const double* x,
                                 const double* fx, const double* lo, const double* hi, double F, double CR,
                                 int strategy, double* u, uint32_t* r_out, uint32_t* jrand_out, uint32_t* take_out,
                                 int* three_point_out, int* best_out) {
  uint32_t cr_thr = CR >= 1.0 ? 0xffffffffu : (uint32_t)(CR * 4294967296.0);
  int cr_all = CR >= 1.0;
  const double K = (F + 1.0) * 0.5;
  /* the previous generation's best (lowest index on ties), for best/1 */
  int best = 0;
  for (int i = 1; i < np; ++i)
    if (fx[i] < fx[best]) best = i;
  if (best_out) *best_out = best;
  for (int i = 0; i < np; ++i) {
    uint32_t w[12], r[3], w4[4];
    oc_draw12(seed, block_id, g, (uint32_t)i, w);
    oc_pick3((uint32_t)i, (uint32_t)np, w, r);
    uint32_t jrand = oc_lemire(w[3], (uint32_t)dim);
    if (strategy == OC_DE_BEST1_JITTER) oc_draw_extra(seed, block_id, g, (uint32_t)i, w4);
    const int three_point = strategy == OC_DE_EITHER_OR && w[9] >= 0x80000000u;
    uint32_t mask = 0;
    for (int j = 0; j < dim; ++j) {
      double parent = x[i * dim + j];
      const double a = x[r[0] * dim + j], b = x[r[1] * dim + j], c = x[r[2] * dim + j];
      double v;
      int take;
      if (strategy == OC_DE_BEST1_JITTER) {
        const uint32_t jw = j < 3 ? w[9 + j] : w4[j - 3];
        const double Fj = F + 1e-4 * ((double)jw * (1.0 / 4294967296.0));
        v = x[best * dim + j] + Fj * (b - c);
        take = (uint32_t)j == jrand || cr_all || w[4 + j] < cr_thr;
      } else if (strategy == OC_DE_EITHER_OR) {
        v = three_point ? a + K * ((b + c) - 2.0 * a) : a + F * (b - c);
        take = 1;
      } else {
        v = a + F * (b - c);
        take = (uint32_t)j == jrand || cr_all || w[4 + j] < cr_thr;
      }
      u[i * dim + j] = take ? oc_repair(j, v, parent, lo, hi) : parent;
      if (take) mask |= 1u << j;
    }
    if (r_out) { r_out[3 * i] = r[0]; r_out[3 * i + 1] = r[1]; r_out[3 * i + 2] = r[2]; }
    if (jrand_out) jrand_out[i] = jrand;
    if (take_out) take_out[i] = mask;
    if (three_point_out) three_point_out[i] = three_point;
  }
}

/* Exported form of one generation's trials for the test suite (the DE loop
 * below calls the same function). bounds: dim (lo, hi) pairs. Returns 0, or
 * -1 on invalid arguments. */
int oc_de_trials(uint64_t seed, uint32_t block_id, uint32_t gen, int np, int dim, const double* x, const double* fx,
                 const double* bounds, double F, double CR, int strategy, double* u, uint32_t* r_out,
                 uint32_t* jrand_out, uint32_t* take_out, int* three_point_out, int* best_out) {
  if (np < 4 || gen < 1 || (dim != OC_D && dim != OC_DF)) return -1;
  if (strategy != OC_DE_RAND1_BIN && strategy != OC_DE_BEST1_JITTER && strategy != OC_DE_EITHER_OR) return -1;
  double lo[OC_DF], hi[OC_DF];
  for (int j = 0; j < dim; ++j) {
    lo[j] = bounds[2 * j];
    hi[j] = bounds[2 * j + 1];
    if (!(lo[j] <= hi[j])) return -1;
  }
  oc_generation_trials(seed, block_id, gen, np, dim, x, fx, lo, hi, F, CR, strategy, u, r_out, jrand_out, take_out,
                       three_point_out, best_out);
  return 0;
}

int oc_de_run_strategy(oc_objective_fn obj, void* user, const double bounds[2 * OC_D], int np, int gens, double F,
                       double CR, uint64_t seed, uint32_t block_id, int strategy, double out[OC_D + 1],
                       double* final_pop, double* final_fit, int nthreads) {
  return oc_de_run_dim(obj, user, OC_D, bounds, np, gens, F, CR, seed, block_id, strategy, out, final_pop, final_fit,
                       nthreads);
}

/* Runs DE/rand/1/bin; returns 0 on success, -1 on invalid arguments.
 * out[0..4] = best vector, out[5] = its objective value.
 * final_pop (np*5) and final_fit (np) are optional. */
int oc_de_run(oc_objective_fn obj, void* user, const double bounds[2 * OC_D], int np, int gens, double F,
              double CR, uint64_t seed, uint32_t block_id, double out[OC_D + 1], double* final_pop,
              double* final_fit, int nthreads) {
  return oc_de_run_strategy(obj, user, bounds, np, gens, F, CR, seed, block_id, OC_DE_RAND1_BIN, out, final_pop,
                            final_fit, nthreads);
}

/* DE over `dim` parameters: 5 for the cubic model, 7 for the full model.
 * Generation 0 draws component j from words 2j and 2j+1 of oc_draw16 (the
 * same words as oc_draw12's for dim 5); later generations draw as for dim 5,
 * with the crossover word of component j at word 4 + j and, for DE/best/1
 * with jitter, the jitter word of component j at word 9 + j (j < 3), else
 * word j - 3 of the fourth counter group. */
int oc_de_run_dim(oc_objective_fn obj, void* user, int dim, const double* bounds, int np, int gens, double F,
                  double CR, uint64_t seed, uint32_t block_id, int strategy, double* out, double* final_pop,
                  double* final_fit, int nthreads) {
  if (np < 4 || gens < 0 || (dim != OC_D && dim != OC_DF)) return -1;
  if (strategy != OC_DE_RAND1_BIN && strategy != OC_DE_BEST1_JITTER && strategy != OC_DE_EITHER_OR) return -1;
  double lo[OC_DF], hi[OC_DF];
  for (int j = 0; j < dim; ++j) {
    lo[j] = bounds[2 * j];
    hi[j] = bounds[2 * j + 1];
    if (!(lo[j] <= hi[j])) return -1;
  }
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  (void)nthreads;
#endif
  double* x = (double*)malloc(sizeof(double) * np * dim);
  double* fx = (double*)malloc(sizeof(double) * np);
  double* u = (double*)malloc(sizeof(double) * np * dim);
  double* fu = (double*)malloc(sizeof(double) * np);
  if (!x || !fx || !u || !fu) { free(x); free(fx); free(u); free(fu); return -1; }

  /* Initial population: uniform inside the bounds (generation index 0). */
  for (int i = 0; i < np; ++i) {
    uint32_t w[16];
    oc_draw16(seed, block_id, 0u, (uint32_t)i, w);
    for (int j = 0; j < dim; ++j) x[i * dim + j] = lo[j] + oc_u53(w[2 * j], w[2 * j + 1]) * (hi[j] - lo[j]);
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int i = 0; i < np; ++i) fx[i] = obj(x + i * dim, user);

  for (int g = 1; g <= gens; ++g) {
    /* mutation + crossover for every individual, from the generation-(g-1) population */
    oc_generation_trials(seed, block_id, (uint32_t)g, np, dim, x, fx, lo, hi, F, CR, strategy, u, NULL, NULL, NULL,
                         NULL, NULL);
    /* evaluate all trials, then select (trial wins ties) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int i = 0; i < np; ++i) fu[i] = obj(u + i * dim, user);
    for (int i = 0; i < np; ++i) {
      if (fu[i] <= fx[i]) {
        memcpy(x + i * dim, u + i * dim, sizeof(double) * dim);
        fx[i] = fu[i];
      }
    }
  }
  int best = 0;
  for (int i = 1; i < np; ++i)
    if (fx[i] < fx[best]) best = i;
  for (int j = 0; j < dim; ++j) out[j] = x[best * dim + j];
  out[dim] = fx[best];
  if (final_pop) memcpy(final_pop, x, sizeof(double) * np * dim);
  if (final_fit) memcpy(final_fit, fx, sizeof(double) * np);
  free(x); free(fx); free(u); free(fu);
  return 0;
}

typedef struct { const double* s; int64_t n; double fs, t0; } oc_block;

static double oc_block_objective(const double* th, void* user) {
  const oc_block* b = (const oc_block*)user;
  return oc_sse(b->s, b->n, b->fs, b->t0, th);
}

static double oc_block_cor_objective(const double* th, void* user) {
  const oc_block* b = (const oc_block*)user;
  return oc_cor_objective(b->s, b->n, b->fs, b->t0, th);
}

/* objective 0: chi-square (Eq. 2-2-4); 1: correlation (Eq. 2-2-5);
 * strategy: OC_DE_RAND1_BIN, OC_DE_BEST1_JITTER or OC_DE_EITHER_OR. */
int oc_de_solve_block_obj(const double* s, int64_t n, double fs, double t0, const double bounds[2 * OC_D], int np,
                          int gens, double F, double CR, uint64_t seed, uint32_t block_id, int objective,
                          int strategy, double out[OC_D + 1], double* final_pop, double* final_fit, int nthreads) {
  if (n < 1 || !(fs > 0.0) || objective < 0 || objective > 1) return -1;
  oc_block b = {s, n, fs, t0};
  return oc_de_run_strategy(objective ? oc_block_cor_objective : oc_block_objective, &b, bounds, np, gens, F, CR,
                            seed, block_id, strategy, out, final_pop, final_fit, nthreads);
}

static double oc_block_full_objective(const double* th, void* user) {
  const oc_block* b = (const oc_block*)user;
  return oc_sse_full(b->s, b->n, b->fs, b->t0, th);
}

/* DE fit of the full model (7 parameters) on the chi-square with one of the
 * strategies (Table 3-1-1 pairs "3" with the chi-square). */
int oc_de_solve_block_full_strategy(const double* s, int64_t n, double fs, double t0, const double bounds[2 * OC_DF],
                                    int np, int gens, double F, double CR, uint64_t seed, uint32_t block_id,
                                    int strategy, double out[OC_DF + 1], double* final_pop, double* final_fit,
                                    int nthreads) {
  if (n < 1 || !(fs > 0.0)) return -1;
  oc_block b = {s, n, fs, t0};
  return oc_de_run_dim(oc_block_full_objective, &b, OC_DF, bounds, np, gens, F, CR, seed, block_id, strategy, out,
                       final_pop, final_fit, nthreads);
}

/* DE/rand/1/bin fit of the full model (7 parameters) on the chi-square. */
int oc_de_solve_block_full(const double* s, int64_t n, double fs, double t0, const double bounds[2 * OC_DF], int np,
                           int gens, double F, double CR, uint64_t seed, uint32_t block_id, double out[OC_DF + 1],
                           double* final_pop, double* final_fit, int nthreads) {
  return oc_de_solve_block_full_strategy(s, n, fs, t0, bounds, np, gens, F, CR, seed, block_id, OC_DE_RAND1_BIN, out,
                                         final_pop, final_fit, nthreads);
}

int oc_de_solve_block(const double* s, int64_t n, double fs, double t0, const double bounds[2 * OC_D], int np,
                      int gens, double F, double CR, uint64_t seed, uint32_t block_id, double out[OC_D + 1],
                      double* final_pop, double* final_fit, int nthreads) {
  return oc_de_solve_block_obj(s, n, fs, t0, bounds, np, gens, F, CR, seed, block_id, 0, OC_DE_RAND1_BIN, out,
                               final_pop, final_fit, nthreads);
}

/* Textbook DE test functions (5-D), for the DE self-check. */
static double oc_sphere(const double* x, void* user) {
  (void)user;
  double s = 0.0;
  for (int j = 0; j < OC_D; ++j) s += x[j] * x[j];
  return s;
}
static double oc_rosenbrock(const double* x, void* user) {
  (void)user;
  double s = 0.0;
  for (int j = 0; j + 1 < OC_D; ++j) {
    double a = x[j + 1] - x[j] * x[j], b = 1.0 - x[j];
    s += 100.0 * a * a + b * b;
  }
  return s;
}

int oc_de_textbook(int which, const double bounds[2 * OC_D], int np, int gens, double F, double CR, uint64_t seed,
                   double out[OC_D + 1]) {
  oc_objective_fn f = which == 0 ? oc_sphere : oc_rosenbrock;
  return oc_de_run(f, NULL, bounds, np, gens, F, CR, seed, 0u, out, NULL, NULL, 1);
}

int oc_de_textbook_strategy(int which, const double bounds[2 * OC_D], int np, int gens, double F, double CR,
                            uint64_t seed, int strategy, double out[OC_D + 1]) {
  oc_objective_fn f = which == 0 ? oc_sphere : oc_rosenbrock;
  return oc_de_run_strategy(f, NULL, bounds, np, gens, F, CR, seed, 0u, strategy, out, NULL, NULL, 1);
}

/* The same textbook functions over `dim` parameters (the dimension rides in
 * `user`), for the DE over the full model's 7 parameters. */
static double oc_sphere_n(const double* x, void* user) {
  const int dim = *(const int*)user;
  double s = 0.0;
  for (int j = 0; j < dim; ++j) s += x[j] * x[j];
  return s;
}
static double oc_rosenbrock_n(const double* x, void* user) {
  const int dim = *(const int*)user;
  double s = 0.0;
  for (int j = 0; j + 1 < dim; ++j) {
    double a = x[j + 1] - x[j] * x[j], b = 1.0 - x[j];
    s += 100.0 * a * a + b * b;
  }
  return s;
}

int oc_de_textbook_dim_strategy(int which, int dim, const double* bounds, int np, int gens, double F, double CR,
                                uint64_t seed, int strategy, double* out) {
  oc_objective_fn f = which == 0 ? oc_sphere_n : oc_rosenbrock_n;
  return oc_de_run_dim(f, &dim, dim, bounds, np, gens, F, CR, seed, 0u, strategy, out, NULL, NULL, 1);
}

int oc_de_textbook_dim(int which, int dim, const double* bounds, int np, int gens, double F, double CR,
                       uint64_t seed, double* out) {
  return oc_de_textbook_dim_strategy(which, dim, bounds, np, gens, F, CR, seed, OC_DE_RAND1_BIN, out);
}

/* ------------------------------------------------------------------------ */
/* Observables in the paper's coefficients c0..c3 (radians). */

/* Eq. 3-1-1: phase and instantaneous frequency (rad, rad/s) at t. */
double oc_c_phase(const double c[4], double t) { return c[0] + c[1] * t + c[2] * t * t + c[3] * t * t * t; }
double oc_c_freq(const double c[4], double t) { return c[1] + 2.0 * c[2] * t + 3.0 * c[3] * t * t; }

/* Eq. 4-1-2 for one block of length T: phi(T/2) - phi(-T/2). */
double oc_c_total_phase(const double c[4], double T) { return oc_c_phase(c, T / 2.0) - oc_c_phase(c, -T / 2.0); }

/* theta = (A, phi0, f0, f1, f2) -> c0..c4 (Eq. 2-2-3 in cycles form). */
void oc_theta_to_c(const double th[OC_D], double c[5]) {
  c[0] = th[1];
  c[1] = 2.0 * OC_PI * th[2];
  c[2] = OC_PI * th[3];
  c[3] = OC_PI * th[4] / 3.0;
  c[4] = th[0];
}
