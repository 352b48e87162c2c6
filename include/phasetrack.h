/*
 * phasetrack -- C ABI of the B300 (sm_103a) implementation of the
 * Differential-Evolution phase-tracking hot path of arxiv 1906.10598
 * ("The GPU-based Phase Tracking method for Planetary Radio Science
 * applications").
 *
 * The paper fits each open-loop tracking block with the Taylor-phase model
 * of Sec. 2.2 Eq. 2-2-2 (amplitude slope c5 = 0), written here in cycles:
 *
 *   m(t) = A cos(2 pi p(t)),   p(t) = phi0/(2 pi) + f0 t + f1 t^2/2 + f2 t^3/6
 *
 * so that c0 = phi0, c1 = 2 pi f0, c2 = pi f1, c3 = pi f2 / 3, c4 = A
 * (Eq. 2-2-3). A candidate is the row theta = (A, phi0, f0, f1, f2) of five
 * doubles. Its objective is the unit-weight chi-square of Eq. 2-2-4,
 *
 *   SSE(theta) = sum_{i=0}^{n-1} (s_i - m(t_i))^2,   t_i = t0 + i / fs,
 *
 * and the fit minimises it by DE (Sec. 1.2 and Table 3-1-1: mutation factor
 * F, crossover CR, a fixed number of iterations as the stop rule).
 *
 * Conventions for every entry point:
 *   - Return value: PT_OK (0) on success, PT_PENDING (1) for a request that
 *     is still running, a negative PT_E* code on failure. No exception or
 *     C++ type crosses this boundary. pt_last_error() describes the last
 *     failure of that context as a NUL-terminated string owned by the context.
 *   - Pointers documented as "host or device" may point to pageable or
 *     pinned host memory or to device memory of the context's GPU; the
 *     library detects which. All such calls are synchronous: when they return,
 *     outputs are written and inputs may be reused.
 *   - Contexts are not thread-safe: one thread at a time per context.
 */
#ifndef PHASETRACK_H
#define PHASETRACK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Entry points are exported from the shared library; everything else is hidden. */
#if defined(__GNUC__)
#define PT_API __attribute__((visibility("default")))
#else
#define PT_API
#endif

typedef struct pt_ctx pt_ctx;

/* Status codes. */
#define PT_OK 0
#define PT_PENDING 1
#define PT_EINVAL (-1)    /* invalid argument (NaN bounds, lo > hi, pop < 4, n < 1, fs <= 0, ...) */
#define PT_ENOMEM (-2)    /* device or host allocation failed */
#define PT_EAGAIN (-3)    /* admission refused: not enough device memory or slots right now */
#define PT_ETIMEOUT (-4)  /* a bounded device-side wait expired; the kernel returned early */
#define PT_ECUDA (-5)     /* a CUDA runtime call failed */
#define PT_ENOTCONV (-6)  /* a result failed its validity check */
#define PT_ENOBLOCK (-7)  /* no block loaded in this context */

/* Sample storage types of pt_load_block (Table "PRSR data recording modes":
 * 8/16-bit quantised narrow-band samples; float types for synthetic data). */
#define PT_I8 0
#define PT_I16 1
#define PT_F16 2
#define PT_F32 3
#define PT_F64 4

/* Precision tiers of the objective.
 *   PT_TIER_F64   (default) phase exact to ~1e-6 rad: per candidate the
 *                 sample-index polynomial is reduced mod one cycle from FP64
 *                 into 128-bit fixed point, re-anchored per 256-sample tile
 *                 with integer arithmetic, walked in 32-bit fixed point;
 *                 FP32 cosine (SFU) and FP32 residuals.
 *   PT_TIER_PLAIN all-FP64 per sample: Horner phase in seconds, FP64
 *                 reduction mod one cycle, FP64 cospi, FP64 residuals.
 *   PT_TIER_DF32  per-sample phase in double-float (pairs of FP32), FP32
 *                 cosine; no FP64 in the sample loop.
 *   PT_TIER_F32   naive FP32 Horner phase in seconds, FP32 cosine. */
#define PT_TIER_F64 0
#define PT_TIER_PLAIN 1
#define PT_TIER_DF32 2
#define PT_TIER_F32 3

/* Objectives (Sec. 2.2), chosen per context with pt_set_objective:
 *   PT_OBJ_CHI2  Eq. 2-2-4 with unit weights, sum_i (s_i - m(t_i))^2 (default);
 *   PT_OBJ_COR   Eq. 2-2-5 with the constant-amplitude model of Eq. 2-2-6,
 *                1 / (atan(cor) + pi/2), cor = sum_i s_i A cos(phi(t_i)), the
 *                unnormalised cross-correlation (the reading under which the
 *                objective tends to 1/pi at the fit, as the paper states).
 *                A is each candidate's amplitude; a DE fit on PT_OBJ_COR
 *                should hold it constant (bounds lo = hi = the average
 *                amplitude), since a free A makes the objective divergent.
 *                Every tier (the sums are s_i cos(phi_i) in each tier's
 *                arithmetic). */
#define PT_OBJ_CHI2 0
#define PT_OBJ_COR 1

/* DE mutation strategies, chosen per context with pt_set_strategy. Table
 * 3-1-1 names the strategy by number only ("3" for Eq. 2-2-4, "6" for
 * Eq. 2-2-5, Sec. 3.1.2), counting six; they are read in the order of
 * Price, Storn & Lampinen (2006), which the paper cites. r1, r2, r3 are the
 * drawn indices (distinct, different from i):
 *   PT_DE_RAND1_BIN     v = x_r1 + F (x_r2 - x_r3), binomial crossover (default);
 *   PT_DE_BEST1_JITTER  "3": v_j = x_best,j + F_j (x_r2,j - x_r3,j) with
 *                       F_j = F + 1e-4 U_j per component, binomial crossover,
 *                       x_best the previous generation's lowest-index minimum;
 *   PT_DE_EITHER_OR     "6": with probability 1/2 the rand/1 mutant, otherwise
 *                       x_r1 + K ((x_r2 + x_r3) - 2 x_r1), K = (F + 1)/2; the
 *                       trial is the mutant itself (no crossover).
 * Out-of-range components are repaired as for the default. */
#define PT_DE_RAND1_BIN 0
#define PT_DE_BEST1_JITTER 3
#define PT_DE_EITHER_OR 6

/* Largest DE population supported by the device kernels. */
#define PT_POP_MAX 128

/* Create a context on CUDA device `device`. The context owns device memory,
 * a CUDA stream and the autotune cache. *out is set on success. */
PT_API int pt_create(pt_ctx** out, int device);

/* Release a context and everything it owns. NULL is allowed. */
PT_API void pt_destroy(pt_ctx* ctx);

/* Description of the last failure on `ctx` (empty string if none). */
PT_API const char* pt_last_error(const pt_ctx* ctx);

/* Use `stream` (a cudaStream_t of the context's device) for all work of this
 * context; NULL restores the context's own stream. The caller keeps ownership. */
PT_API int pt_set_stream(pt_ctx* ctx, void* stream);

/* The cudaStream_t the context launches on. */
PT_API void* pt_get_stream(const pt_ctx* ctx);

/* Load one data block (Sec. 2.2: a contiguous block of n samples with the
 * time origin t0 of sample 0; a block centred on 0 has t0 = -(n-1)/(2 fs)).
 *   samples  host or device pointer to n values of type `dtype`; copied, so
 *            the caller keeps ownership.
 *   n        number of samples, n >= 1.
 *   dtype    PT_I8, PT_I16, PT_F16, PT_F32 or PT_F64.
 *   scale    physical value of sample i is scale * samples[i] (scale > 0).
 *   fs       sampling rate in Hz (> 0); t_i = t0 + i / fs.
 * Replaces the context's current block. Errors: PT_EINVAL, PT_ENOMEM, PT_ECUDA. */
PT_API int pt_load_block(pt_ctx* ctx, const void* samples, int64_t n, int dtype, double scale, double fs, double t0);

/* Objective of the context's later pt_objective, pt_de_solve[_ex], pt_track
 * and pt_batch calls, and of its serving loop, which takes the objective and
 * the strategy in force when it starts (its first pt_submit): PT_OBJ_CHI2
 * (default) or PT_OBJ_COR. Values returned as "sse" are then the objective
 * value. Errors: PT_EINVAL. */
PT_API int pt_set_objective(pt_ctx* ctx, int objective);

/* DE strategy of the context's later pt_de_solve[_ex], pt_track and
 * pt_batch calls, and of its serving loop when it starts: PT_DE_RAND1_BIN (default), PT_DE_BEST1_JITTER or
 * PT_DE_EITHER_OR. Errors: PT_EINVAL. */
PT_API int pt_set_strategy(pt_ctx* ctx, int strategy);

/* Evaluate Eq. 2-2-4 for n candidates on the loaded block.
 *   cands    host or device pointer, n rows of 5 doubles (A, phi0, f0, f1, f2), row-major.
 *   sse_out  host or device pointer, n doubles.
 *   tier     PT_TIER_*.
 * The result is deterministic: it does not depend on the launch shape.
 * Errors: PT_EINVAL, PT_ENOBLOCK, PT_ENOMEM, PT_ECUDA, PT_ETIMEOUT. */
PT_API int pt_objective(pt_ctx* ctx, const double* cands, int64_t n, double* sse_out, int tier);

/* Fit the loaded block by DE (Sec. 1.2, Table 3-1-1; the context's strategy,
 * DE/rand/1/bin by default, and objective) in one persistent device launch.
 *   bounds      host pointer, 5 x 2 doubles: (lo, hi) per parameter. The phi0
 *               range wraps when it spans a full circle (Sec. 3.1.1: [0, 2 pi]);
 *               other out-of-range trial components move to the midpoint of
 *               the violated bound and the parent's component.
 *   pop         population size, 4 <= pop <= PT_POP_MAX.
 *   gens        generations after the initial population (itermax), >= 0.
 *   F, CR       mutation factor and crossover rate (CR >= 1 crosses every component).
 *   seed        Philox4x32-10 key; the draws of individual i at generation g
 *               use counters (k, i, g, block_id), k = 0, 1, 2 (block_id 0 here).
 *   params_out  host or device pointer, 6 doubles: best (A, phi0, f0, f1, f2)
 *               and its SSE; written only on success. Ties go to the lowest index.
 *   tier        PT_TIER_*.
 * Errors: PT_EINVAL, PT_ENOBLOCK, PT_ENOMEM, PT_ECUDA, PT_ETIMEOUT. */
PT_API int pt_de_solve(pt_ctx* ctx, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                double* params_out, int tier);

/* pt_de_solve with a Philox block id and the final population:
 *   pop_out  optional (NULL) host or device pointer, pop x 5 doubles.
 *   fit_out  optional (NULL) host or device pointer, pop doubles (their SSE). */
PT_API int pt_de_solve_ex(pt_ctx* ctx, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                   uint32_t block_id, double* params_out, double* pop_out, double* fit_out, int tier);

/* ---- The full model -------------------------------------------------------
 * Eq. 2-2-2 with the amplitude slope c5 and the Taylor phase of Eq. 2-2-1 at
 * order n = 4 (Sec. 3.2, for high-dynamics arcs near perigee), 7 parameters
 * theta = (A, phi0, f0, f1, f2, A1, f3):
 *   m(t) = (A + A1 t) cos(phi0 + 2 pi (f0 t + f1 t^2/2 + f2 t^3/6 + f3 t^4/24)),
 * i.e. c4 = A, c5 = A1 and the order-4 phase coefficient f3 (cycles/s^4). The
 * chi-square of Eq. 2-2-4 only (Eq. 2-2-5's model has a constant amplitude):
 * the full-model calls fail with PT_EINVAL unless the context's objective is
 * PT_OBJ_CHI2. Every precision tier and DE strategy applies (the paper's own setting is Dim_XC = 6 with strategy
 * "3"). A parameter held at lo = hi stays there, so A1 = 0 or f3 = 0 gives
 * the 6-parameter forms. */

/* Evaluate Eq. 2-2-4 of the full model for n candidates on the loaded block.
 *   cands    host or device pointer, n rows of 7 doubles, row-major.
 *   sse_out  host or device pointer, n doubles.
 *   tier     PT_TIER_* (the default tier's phase re-expansion carries the
 *            quartic term; the others evaluate the quartic Horner form).
 * Deterministic (independent of the launch shape).
 * Errors: PT_EINVAL, PT_ENOBLOCK, PT_ENOMEM, PT_ECUDA, PT_ETIMEOUT. */
PT_API int pt_objective_full(pt_ctx* ctx, const double* cands, int64_t n, double* sse_out, int tier);

/* Fit the loaded block with the full model by the context's DE strategy, as
 * pt_de_solve_ex over 7 parameters. The draws are pt_de_solve_ex's, with the
 * generation-0 words 12 and 13 of component 6 from counter (3, i, 0, block_id),
 * the crossover words of components 5, 6 at words 9, 10 and (PT_DE_BEST1_JITTER)
 * their jitter words at words 2, 3 of counter (3, i, g, block_id).
 *   bounds      host pointer, 7 x 2 doubles.
 *   params_out  host or device pointer, 8 doubles: the best theta and its SSE.
 *   pop_out     optional host or device pointer, pop x 7 doubles.
 *   fit_out     optional host or device pointer, pop doubles.
 *   tier        PT_TIER_*.
 * Errors: PT_EINVAL, PT_ENOBLOCK, PT_ENOMEM, PT_ECUDA, PT_ETIMEOUT. */
PT_API int pt_de_solve_full(pt_ctx* ctx, const double* bounds, int pop, int gens, double F, double CR, uint64_t seed,
                            uint32_t block_id, double* params_out, double* pop_out, double* fit_out, int tier);

/* ---- Batched fits ---------------------------------------------------------
 * Many independent blocks of uneven length, each with its own DE controls and
 * population, solved in one persistent cooperative launch (replayed from a
 * captured CUDA graph when the driver allows it). The paper fits its blocks
 * one after another (Sec. 3.1.4, data process flow); a batch runs them
 * concurrently. A block's result is bit-identical to pt_de_solve_ex on the
 * same block alone: its sums of squares are exact integer sums of the same
 * per-tile partials whatever CTAs evaluate them. */

/* One block of a batch: the data block of Sec. 2.2 and the DE controls of
 * Table 3-1-1 (meanings as in pt_load_block and pt_de_solve_ex). */
typedef struct pt_block_spec {
  const void* samples; /* host or device pointer, n values of type dtype; copied by pt_batch_create */
  int64_t n;
  int dtype;
  double scale, fs, t0;
  double bounds[10]; /* (lo, hi) for A, phi0, f0, f1, f2 */
  int pop, gens;
  double F, CR;
  uint64_t seed;
  uint32_t block_id;
} pt_block_spec;

/* Result of one fit: the best (A, phi0, f0, f1, f2) and its SSE. */
typedef struct pt_fit {
  double params[5];
  double sse;
} pt_fit;

typedef struct pt_batch pt_batch;

typedef struct pt_batch_info {
  int nblocks;
  int ngroups;      /* groups of CTAs working concurrently */
  int group_ctas;   /* CTAs per group (per block in flight) */
  int tier;
  int uses_graph;   /* 1 if pt_batch_run replays a captured CUDA graph */
  double sample_evals;  /* sum over blocks of n * pop * (gens + 1) */
  double predicted_ms;  /* the autotuner's makespan estimate */
  double last_ms;       /* device time of the last pt_batch_run */
  double tune_rate;     /* calibrated objective sample-evals/s per CTA, tiles resident */
  double tune_gen_us;   /* calibrated fixed cost per generation (us) */
  double tune_rate_stream; /* calibrated sample-evals/s per CTA, tiles staged chunk by chunk */
} pt_batch_info;

/* Copy the blocks to the device, choose the launch shape and capture it.
 *   group_ctas  CTAs per block in flight; 0 lets the autotuner choose: it
 *               calibrates the per-CTA rate and the per-generation costs on
 *               the batch's first block (cached in the context) and picks the
 *               group size whose longest-processing-time schedule of the
 *               blocks over the groups has the shortest predicted makespan.
 * Errors: PT_EINVAL, PT_ENOMEM, PT_ECUDA. *out is owned by the caller. */
PT_API int pt_batch_create(pt_ctx* ctx, const pt_block_spec* specs, int nblocks, int tier, int group_ctas,
                           pt_batch** out);

/* A batch of full-model fits (pt_de_solve_full: amplitude slope and order-4
 * phase, chi-square; PT_EINVAL otherwise) in the given tier:
 * specs[i].bounds holds block i's first five (lo, hi) pairs and
 * ext_bounds[4 i .. 4 i + 3] its A1 and f3 pairs (host pointer, nblocks x 4).
 * The autotuner calibrates on the full model (its cache records the model).
 * Results: pt_batch_results_full (pt_batch_results gives the first five). */
PT_API int pt_batch_create_full(pt_ctx* ctx, const pt_block_spec* specs, const double* ext_bounds, int nblocks,
                                int tier, int group_ctas, pt_batch** out);

/* Solve every block of the batch (synchronous). Errors: PT_ECUDA, PT_ETIMEOUT. */
PT_API int pt_batch_run(pt_batch* batch);

/* Copy the results of the last run: out holds nblocks entries (host pointer). */
PT_API int pt_batch_results(pt_batch* batch, pt_fit* out);

/* The results of the last run as nblocks rows of 8 doubles (host pointer):
 * (A, phi0, f0, f1, f2, A1, f3) and the SSE; A1 = f3 = 0 for a cubic batch. */
PT_API int pt_batch_results_full(pt_batch* batch, double* out);

PT_API int pt_batch_get_info(const pt_batch* batch, pt_batch_info* info);

/* Release the batch's device memory and graph. NULL is allowed. */
PT_API void pt_batch_destroy(pt_batch* batch);

/* ---- Serving: station streams, continuous batching -------------------------
 * Blocks arrive from several station streams as they fill (Sec. 3.1.4: the
 * software processes the data stream block by block without manual
 * intervention). pt_submit queues a block and returns at once; a worker
 * thread of the context admits queued blocks into device slots as slots and
 * device memory free up, each admitted block running on its own CUDA stream
 * so its work overlaps the others already on the device; pt_poll collects a
 * finished fit. A block's fit is bit-identical to pt_de_solve_ex on the same
 * block alone, whatever else is in flight. */

/* Models of a served request. */
#define PT_MODEL_CUBIC 0 /* (A, phi0, f0, f1, f2): block.bounds */
#define PT_MODEL_FULL 1  /* the full model of pt_de_solve_full: block.bounds, then ext_bounds for A1, f3 */

typedef struct pt_request {
  pt_block_spec block; /* samples are copied by pt_submit */
  int tier;            /* PT_TIER_* */
  int stream_id;       /* caller's station-stream id, returned in the result */
  int model;           /* PT_MODEL_CUBIC (0, the default of a zeroed request) or PT_MODEL_FULL */
  double ext_bounds[4]; /* PT_MODEL_FULL: (lo, hi) for A1 and f3 */
} pt_request;

typedef struct pt_result {
  pt_fit fit;
  int status;          /* PT_OK, or the error the fit ended with */
  int stream_id;
  double t_submit;     /* seconds on the library's monotonic clock (pt_clock) */
  double t_admit;      /* when the block started on the device */
  double t_done;       /* when the worker saw the fit complete */
  double ext_params[2]; /* PT_MODEL_FULL: the fit's A1 and f3 (0 otherwise) */
} pt_result;

/* Configure the serving loop (before the first pt_submit; later calls fail
 * with PT_EINVAL while requests are in flight):
 *   max_inflight      blocks on the device at once (1..32)
 *   ctas_per_request  CTAs of each block's cooperative launch; 0 = SMs / max_inflight
 *   mem_budget_bytes  device memory the slots may hold; 0 = half of the free memory
 *   max_queued        blocks waiting for a slot before pt_submit returns PT_EAGAIN */
PT_API int pt_serve_configure(pt_ctx* ctx, int max_inflight, int ctas_per_request, int64_t mem_budget_bytes,
                              int max_queued);

/* Queue one block. Returns PT_OK and a ticket, PT_EAGAIN when the queue is
 * full (retry after pt_poll has collected results), or PT_EINVAL (bad
 * arguments, or a block larger than the memory budget). Non-blocking. */
PT_API int pt_submit(pt_ctx* ctx, const pt_request* req, uint64_t* ticket);

/* PT_OK and the result (which is then released), PT_PENDING while queued or
 * running, PT_EINVAL for an unknown ticket. Non-blocking. */
PT_API int pt_poll(pt_ctx* ctx, uint64_t ticket, pt_result* out);

/* Seconds on the monotonic clock used by pt_result. */
PT_API double pt_clock(void);

/* ---- Block-to-block tracking helpers (host only) ---------------------------
 * Running-time range setting of Sec. 3.1.1: the ranges for block n+1 are
 * extrapolated from block n's fit. prev is (A, phi0, f0, f1, f2) of block n
 * about its centre; dt is the time from block n's centre to block n+1's
 * centre; T_next the length of block n+1. Output bounds (5 x 2):
 *   A     +-10 % of A;
 *   phi0  the full circle [-pi, pi);
 *   f0    the instantaneous frequency (Eq. 3-1-1) between the shared border
 *         and the far end of block n+1, widened by min_f0 on each side;
 *   f1    the frequency rate over the same span, widened by min_f1;
 *   f2    f2 +- min_f2 (the paper narrows c3 after the first fit).
 * min_* <= 0 take 2/T_next, 4/T_next^2, 24/T_next^3. */
PT_API int pt_warm_bounds(const double prev[5], double dt, double T_next, double min_f0, double min_f1,
                          double min_f2, double bounds_out[10]);

/* Continuity check of Eq. 3-1-2: the phase (mod 2 pi) and frequency of block
 * a (length Ta, about its centre) at its right border against block b
 * (length Tb, about its own centre) at its left border; the two borders are
 * the same instant for contiguous blocks.
 * Writes |dphi| (rad, wrapped to [0, pi]) and |dF| (rad/s); returns 1 if both
 * are within the thresholds, 0 if not, PT_EINVAL for bad arguments. */
PT_API int pt_continuity(const double a[5], double Ta, const double b[5], double Tb, double max_dphi,
                         double max_dfreq, double* dphi, double* dfreq);

/* Running-time ranges of the full model (7 parameters, see pt_de_solve_full)
 * for block n+1 from block n's fit `prev`, as pt_warm_bounds with the phase
 * carried to order 4: the f0, f1 and f2 ranges span the frequency
 * f0 + f1 t + f2 t^2/2 + f3 t^3/6, its rate f1 + f2 t + f3 t^2/2 and
 * f2 + f3 t over block n+1 (at least +-2/T, +-4/T^2, +-24/T^3 about their
 * centre values), f3 +- 192/T^4 about prev's (about +-pi rad at the block
 * edge, as f2's +-24/T^3 in the cubic model), A +- 10 % about the amplitude
 * extrapolated to block n+1's centre, phi0 over the full circle, and A1 over
 * a1_range (Sec. 3.1.1: "the range of c5 can be fixed"; NULL: prev's A1
 * +- 0.2 A / T). bounds_out: 7 (lo, hi) pairs. Errors: PT_EINVAL. */
PT_API int pt_warm_bounds_full(const double prev[7], double dt, double T_next, const double a1_range[2],
                               double bounds_out[14]);

/* pt_continuity for full-model fits: the border phase and frequency carry the
 * f3 t^4/24 term. Returns 1, 0 or PT_EINVAL as pt_continuity. */
PT_API int pt_continuity_full(const double a[7], double Ta, const double b[7], double Tb, double max_dphi,
                              double max_dfreq, double* dphi, double* dfreq);

/* ---- Initial ranges from FFTs ------------------------------------------------
 * Sec. 3.1.1: the first block's ranges come from an FFT of a small piece of
 * data at the block centre (c1 and c4), a central difference of three
 * frequencies near the centre (c2), and fixed ranges for c3 and c5. Here:
 * three pieces of piece_len samples (0: the largest power of two <= n/4, at
 * most 8192) starting at n/2 - piece_len/2 + (k - 1) piece_len, k = 0, 1, 2;
 * a periodic Hann window; the peak of |X|^2 over bins 1 .. piece_len/2 - 1
 * (lowest index on ties; positive frequencies, as a real tone cannot tell f0
 * from -f0), refined by a parabola through the log magnitudes of the peak and
 * its neighbours; each piece's frequency taken at its sample piece_len/2. */
typedef struct pt_seed_result {
  double f0;               /* frequency at t = 0 (Hz), from the centre piece and f1 */
  double f1;               /* frequency rate (Hz/s), central difference of the outer pieces */
  double A;                /* amplitude from the centre piece's peak, corrected by the window's response */
  int piece_len;
  int peak_bin[3];         /* each piece's peak bin */
  double peak_delta[3];    /* its refined offset (bins) */
  double piece_freq[3];    /* (peak_bin + peak_delta) fs / piece_len (Hz) */
  double piece_time[3];    /* time of each piece's sample piece_len/2 (s) */
  double bounds[14];       /* 7 (lo, hi) pairs: A, phi0, f0, f1, f2, A1, f3 (the first 5: the cubic model) */
} pt_seed_result;

/* Seed the loaded block's ranges: A and f0 +- f0_rel (the paper: 0.1) of their
 * estimates, phi0 the full circle, f1 +- max(f0_rel |f1|, fs^2/piece_len^2)
 * (the paper gives no f1 range: one bin over the pieces' spacing), f2 over
 * c3 = pi f2 / 3 in [-50, 50] rad/s^3, A1 +- 0.2 A / T (T = n / fs) and f3
 * +- 192 / T^4 (about +- pi rad at the block edge; the paper gives none).
 * f0_rel in (0, 1), piece_len 0 or a power of two in [16, 8192] with three
 * pieces inside the block. Errors: PT_EINVAL, PT_ENOBLOCK, PT_ECUDA. */
PT_API int pt_seed_bounds(pt_ctx* ctx, double f0_rel, int piece_len, pt_seed_result* out);

/* ---- Block-to-block tracking of one stream ----------------------------------
 * The data process flow of Sec. 3.1.4 for one station stream cut into
 * contiguous blocks, each fitted about its own centre (t0 = -(n-1)/(2 fs)):
 *   - ranges: the first block takes the session's initial bounds; each later
 *     block takes the running-time ranges of Sec. 3.1.1 (pt_warm_bounds)
 *     extrapolated from the last accepted fit over the time between centres;
 *   - acceptance: the continuity check of Eq. 3-1-2 (pt_continuity) against
 *     the previous block when that block was accepted (the first block, and a
 *     block after an abandoned one, have no adjacent reference and are
 *     accepted unchecked);
 *   - retry: a rejected fit is searched again with the f0, f1, f2 half-widths
 *     multiplied by `enlarge` and A widened by the same factor (phi0 keeps the
 *     full circle), with a new DE seed; after `max_attempts` searches the
 *     block is abandoned (the paper abandons it after three, Sec. 3.1.4);
 *   - observables: the border phase and frequency (Eq. 3-1-2), the block's
 *     total phase phi(T/2) - phi(-T/2) and, over each count interval T_c of
 *     accepted contiguous blocks, the integration Doppler
 *     Phi_total / T_c (Eq. 4-1-2); an abandoned block breaks the interval.
 * The paper's output record (Appendix 1) carries a data quality index it does
 * not define; here it is the number of the search that was accepted (1 = the
 * first), or 0 for an abandoned block. */
typedef struct pt_track pt_track;

typedef struct pt_track_config {
  int pop, gens;           /* DE controls of every search (Table 3-1-1) */
  double F, CR;
  uint64_t seed;           /* search k of block i uses Philox key seed + k, block id i */
  int tier;                /* PT_TIER_* */
  double max_dphi;         /* continuity threshold on the border phase (rad), > 0 */
  double max_dfreq;        /* continuity threshold on the border frequency (rad/s), > 0 */
  double enlarge;          /* range factor per retry, >= 1 */
  int max_attempts;        /* searches per block, >= 1 (the paper: 3) */
  double count_interval;   /* T_c of the integration Doppler (s); <= 0 disables it */
} pt_track_config;

typedef struct pt_track_result {
  int64_t block_index;     /* 0, 1, ... in submission order */
  int quality;             /* accepted search (1..max_attempts), 0 = abandoned */
  int attempts;            /* searches made for this block */
  double params[7];        /* accepted (A, phi0, f0, f1, f2, A1, f3) about the block centre; the last search's if
                              abandoned; A1 = f3 = 0 in a cubic-model session */
  double sse;
  double dphi, dfreq;      /* continuity residuals of the accepted search (NaN if unchecked) */
  double phi_left, phi_right;  /* border phase mod 2 pi (rad) at -T/2 and T/2 */
  double f_left, f_right;      /* border frequency (rad/s) */
  double total_phase;      /* phi(T/2) - phi(-T/2) (rad), the Eq. 4-1-2 term; NaN if abandoned */
  double int_doppler;      /* Phi_total / T_c (rad/s) when this block completes a count interval, else NaN */
  double interval_phase;   /* Phi_total of that interval (rad), else NaN */
  double bounds[14];       /* (lo, hi) pairs of the last search's ranges: A, phi0, f0, f1, f2[, A1, f3]
                              (the last 4 entries are 0 in a cubic-model session) */
} pt_track_result;

/* Start a session on ctx (which it uses for every fit; one session per
 * context at a time). bounds: the first block's (lo, hi) pairs for A, phi0,
 * f0, f1, f2 (host pointer, 10 doubles), lo <= hi; a parameter whose range is
 * a point (lo == hi) stays at that value in every search of the session (the
 * constant amplitude of the correlation objective, Eq. 2-2-6, or f3 = 0 for
 * the paper's 6-parameter model in a full-model session).
 * Errors: PT_EINVAL, PT_ENOMEM. */
PT_API int pt_track_create(pt_ctx* ctx, const pt_track_config* cfg, const double bounds[10], pt_track** out);

/* A session that fits every block with the full model (pt_de_solve_full:
 * amplitude slope and order-4 phase, for arcs near perigee, Sec. 3.2):
 * bounds holds 7 (lo, hi) pairs; later blocks take pt_warm_bounds_full with
 * the initial A1 range, acceptance uses pt_continuity_full, and a retry also
 * widens the f3 range. The context must be on the chi-square (the fits
 * fail with PT_EINVAL otherwise). Errors: PT_EINVAL, PT_ENOMEM. */
PT_API int pt_track_create_full(pt_ctx* ctx, const pt_track_config* cfg, const double bounds[14], pt_track** out);

/* Fit the stream's next block (samples as in pt_load_block, the context's
 * current block is replaced), synchronously; *out is always written when the
 * return is PT_OK, which it is also for an abandoned block (quality 0).
 * Errors: PT_EINVAL (bad arguments), and those of pt_load_block and
 * pt_de_solve_ex, which leave the session unchanged. */
PT_API int pt_track_block(pt_track* tr, const void* samples, int64_t n, int dtype, double scale, double fs,
                          pt_track_result* out);

PT_API void pt_track_destroy(pt_track* tr);

/* ---- Objective without allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for host
 * programs that must not allocate device memory on their call path, such as
 * a real-time recording pipeline that reserves the GPU's memory up front in
 * its own pool, or a framework that forbids driver allocations after
 * start-up. It computes what pt_objective computes without a context and
 * without calling cudaMalloc, cudaFree or any allocating routine:
 *   - every input and output is a device buffer the caller owns;
 *   - the only scratch is a fixed array in the library's device memory
 *     (PT_NOALLOC_MAX_CANDIDATES + 32 64-bit words, about 33 KB), which every
 *     GPU that loads the library holds until the process exits.
 * Arguments:
 *   samples   device pointer, 16-byte aligned, to ceil(n/256)*256 readable
 *             values of type dtype inside one allocation (values past n are
 *             read and ignored): the tiles are staged by bulk copies that need
 *             16-byte-aligned sources and read whole 256-sample tiles.
 *   n, dtype, scale, fs, t0  as in pt_load_block.
 *   smax      an upper bound on |scale * sample|; 0 takes the type's range
 *             (128, 32768, 65504 times scale for I8, I16, F16). F32 and F64
 *             samples need an explicit bound. The per-tile sums are fixed
 *             point scaled so that n (smax + |A|)^2 fits 61 bits, so a loose
 *             bound coarsens them: pass a tight one (the type's range is
 *             tight for integer samples quantised to their full range, not
 *             for FP16 samples of a few units).
 *   cands     device pointer, 8-byte aligned, ncand rows of 5 doubles (A, phi0,
 *             f0, f1, f2) inside one allocation.
 *   ncand     1 <= ncand <= PT_NOALLOC_MAX_CANDIDATES; larger is PT_EINVAL.
 *   sse_out   device pointer, 8-byte aligned, ncand doubles inside one
 *             allocation.
 * Every buffer must be memory of the current device (or managed memory).
 *   tier      PT_TIER_*.
 *   stream    cudaStream_t to launch on (NULL: the legacy default stream).
 * The call is synchronous on `stream`. The first call on a device looks up
 * the scratch array's device address with that device current and caches it;
 * make that first call before any stream capture. Every call clears the
 * scratch before use (the array keeps the previous call's contents); calls
 * whose work overlaps on the GPU share the one array and race, so callers must
 * serialise them (one stream, or one call at a time per device).
 * Errors: PT_EINVAL (sizes; a pointer that is not memory of the current
 * device, is misaligned, or whose span runs past the end of its allocation,
 * found on the host before anything is launched; a missing bound), PT_ECUDA,
 * PT_ETIMEOUT. */
#define PT_NOALLOC_MAX_CANDIDATES 4096
PT_API int pt_objective_noalloc(const void* samples, int64_t n, int dtype, double scale, double fs, double t0,
                                double smax, const double* cands, int64_t ncand, double* sse_out, int tier,
                                void* stream);

/* ---- Pipe rates of this GPU (the objective's roofline denominators) --------
 * The paper has no counterpart: it reports times, not pipe rates. The
 * objective issues one SFU cosine per sample-evaluation beside a few FP32
 * FMA-pipe instructions, and the DE's trial generation runs on the FP64 pipe;
 * these microbenchmarks measure those pipes on the device in use, with one
 * CTA of 1024 threads per SM running independent chains:
 *   PT_PIPE_COS   __cosf back to back, each with `nffma` (0, 2, 4, 6 or 8)
 *                 further FP32 FMAs on other registers;
 *   PT_PIPE_FFMA  FP32 FMAs alone (nffma ignored);
 *   PT_PIPE_DFMA  FP64 FMAs alone (nffma ignored);
 *   PT_PIPE_EX2   ex2.approx back to back, another SFU function, for
 *                 comparison with the cosine (nffma ignored).
 * Outputs (host pointers): *per_clk_sm = operations (cosines, or FMAs) per SM
 * clock per SM, from clock64 counts between CTA barriers (median over SMs);
 * *per_s = operations per second over the whole GPU (CUDA events);
 * *sm_mhz = the SM clock those two imply. Best of five launches after one
 * untimed launch; the call is synchronous on the legacy default stream, makes
 * `device` current, and allocates and frees a few KB of device memory.
 * Errors: PT_EINVAL (kind, nffma, device, null outputs), PT_ECUDA. */
#define PT_PIPE_COS 0
#define PT_PIPE_FFMA 1
#define PT_PIPE_DFMA 2
#define PT_PIPE_EX2 3
PT_API int pt_pipe_rate(int device, int kind, int nffma, double* per_clk_sm, double* per_s, double* sm_mhz);

/* Device time in milliseconds of the last pt_objective / pt_de_solve kernel
 * work, measured with CUDA events on the context's stream. */
PT_API int pt_last_kernel_ms(const pt_ctx* ctx, float* ms);

/* Limit of every bounded device-side wait of this context's launches (the
 * bulk-copy completion and the DE exchange's arrival polls), in seconds,
 * 1e-3 .. 60 (default 2). A wait that runs out sets the launch's error word,
 * every CTA returns, and the call reports PT_ETIMEOUT; the context stays
 * usable. Errors: PT_EINVAL. */
PT_API int pt_set_wait_timeout(pt_ctx* ctx, double seconds);

/* Failure injection for tests of the bounded waits, host side: while enabled,
 * the context's DE launches start one CTA fewer than the group size the
 * kernel is told, so the last rank's arrivals never come and every
 * exchange wait runs out after the wait limit (PT_ETIMEOUT). No fault, trap
 * or unbounded wait is involved. Errors: PT_EINVAL. */
PT_API int pt_inject_missing_cta(pt_ctx* ctx, int enable);

/* Failure injection for the test of the sample-staging wait, host side: while
 * enabled, the context's objective and DE launches tell each CTA's staging
 * mbarrier to expect 16 bytes more than its bulk copies bring (no extra copy,
 * no other address), so that wait cannot complete and runs out after the wait
 * limit; the CTA then accounts for the 16 bytes itself, waits (bounded) for
 * the copies that did run, and returns, and the call reports PT_ETIMEOUT.
 * The context stays usable. Errors: PT_EINVAL. */
PT_API int pt_inject_short_tx(pt_ctx* ctx, int enable);

#ifdef __cplusplus
}
#endif

#endif /* PHASETRACK_H */
