"""Pins of the oracle's DE one-step rules (Sec. 1.2 mutation -> crossover ->
selection, with the Table 3-1-1 controls F and CR, and the readings of the
paper's silent points: index draws, binomial crossover, bound repair, and the
strategies "3" and "6").

Each test fails on a plausible misreading of one rule:
* index draws: r1, r2, r3 distinct and different from i, each word mapped by
  Lemire's multiply-shift onto the remaining indices in ascending order, so
  every allowed index is reached by exactly the words that mapping gives it
  (checked at every step edge of the word range);
* crossover: the mutant's component is taken with probability CR (binomial
  bound), component jrand always, every component at CR = 1, only jrand at
  CR = 0;
* repair: a component pushed below (above) its range lands exactly on the
  midpoint of the bound and the parent; phi0 on a full-circle range wraps by
  whole turns;
* strategy "6": the three-point coin is fair (binomial bound) and no
  crossover is applied; strategy "3": the jitter factor lies in
  [F, F + 1e-4) and the base is the previous generation's lowest-index
  minimum.
Finally a short restatement of one generation written from those
definitions (words from the Philox generator, pinned by its known answers
elsewhere; index draws by removal from a list rather than by shifting past
sorted exclusions) must give the oracle's trial vectors bit for bit.
"""
import math

import numpy as np
import pytest

import oracle

TWO32 = 1 << 32


def _edges(k):
    """w_v = ceil(v 2^32 / k): the first word Lemire's mapping sends to v."""
    return [(v * TWO32 + k - 1) // k for v in range(k)]


@pytest.mark.parametrize("np_", [4, 5, 17, 128])
def test_index_draws_follow_lemire_onto_remaining_indices(np_):
    rng = np.random.default_rng(np_)
    ivals = range(np_) if np_ <= 17 else [0, 1, 63, 64, 126, 127]
    for i in ivals:
        allowed = [j for j in range(np_) if j != i]
        # first draw: every step edge of the word range
        for v, w in enumerate(_edges(np_ - 1)):
            assert oracle.pick3(i, np_, [w, 0, 0])[0] == allowed[v]
            if v:
                assert oracle.pick3(i, np_, [w - 1, 0, 0])[0] == allowed[v - 1]
        assert oracle.pick3(i, np_, [TWO32 - 1, 0, 0])[0] == allowed[-1]
        # second and third draws, after a random first (and second) pick
        w0 = int(rng.integers(0, TWO32))
        r1 = allowed[(w0 * (np_ - 1)) >> 32]
        rest = [j for j in allowed if j != r1]
        for v, w in enumerate(_edges(np_ - 2)):
            assert oracle.pick3(i, np_, [w0, w, 0])[1] == rest[v]
            if v:
                assert oracle.pick3(i, np_, [w0, w - 1, 0])[1] == rest[v - 1]
        w1 = int(rng.integers(0, TWO32))
        r2 = rest[(w1 * (np_ - 2)) >> 32]
        rest2 = [j for j in rest if j != r2]
        for v, w in enumerate(_edges(np_ - 3)):
            assert oracle.pick3(i, np_, [w0, w1, w])[2] == rest2[v]
            if v:
                assert oracle.pick3(i, np_, [w0, w1, w - 1])[2] == rest2[v - 1]


@pytest.mark.parametrize("np_", [4, 5, 17, 128])
def test_index_draws_distinct_and_exact_multiplicity(np_):
    rng = np.random.default_rng(100 + np_)
    for _ in range(2000):
        i = int(rng.integers(0, np_))
        r = oracle.pick3(i, np_, rng.integers(0, TWO32, 3, dtype=np.uint64).astype(np.uint32))
        assert len({i, *map(int, r)}) == 4
        assert all(0 <= v < np_ for v in r)
    # the multiplicity of each allowed index for the first draw: the words
    # between consecutive step edges, floor or ceil of 2^32 / (np - 1), summing to 2^32
    e = _edges(np_ - 1) + [TWO32]
    counts = [b - a for a, b in zip(e, e[1:])]
    assert sum(counts) == TWO32
    assert set(counts) <= {TWO32 // (np_ - 1), -(-TWO32 // (np_ - 1))}


def _population(rng, pop, bounds):
    lo, hi = bounds[:, 0], bounds[:, 1]
    return lo + rng.random((pop, bounds.shape[0])) * (hi - lo)


BOUNDS5 = np.array([[0.5, 2.0], [-math.pi, math.pi], [-3.0, 3.0], [-1.0, 1.0], [-0.1, 0.1]])


# ranges no mutant of a _population(rng, pop, BOUNDS5) leaves, and phi0's
# below a full circle, so no repair applies: the trial is the mutant itself
WIDE = np.array([[-1e6, 1e6], [-3.0, 3.0], [-1e6, 1e6], [-1e6, 1e6], [-1e6, 1e6]])


def _narrow_phase(x):
    x = x.copy()
    x[:, 1] *= 0.5 / math.pi  # phi0 within [-0.5, 0.5]: mutants stay inside WIDE's [-3, 3]
    return x


def _rand1_mutants(x, r, F):
    """v = x_r1 + F (x_r2 - x_r3) for every individual (DE/rand/1)."""
    a, b, c = x[r[:, 0]], x[r[:, 1]], x[r[:, 2]]
    return a + F * (b - c)


@pytest.mark.parametrize("CR", [0.0, 0.3, 0.9, 1.0])
def test_crossover_takes_mutant_at_rate_cr_and_always_jrand(CR):
    rng = np.random.default_rng(7)
    pop, dim = 128, 5
    n_other, n_taken = 0, 0
    for g in range(1, 41):
        x = _population(rng, pop, BOUNDS5)
        fx = rng.random(pop)
        t = oracle.de_trials(11, 3, g, x, fx, BOUNDS5, 0.5, CR)
        for i in range(pop):
            m, jr = int(t["take"][i]), int(t["jrand"][i])
            assert (m >> jr) & 1
            for j in range(dim):
                taken = (m >> j) & 1
                if not taken:
                    assert t["u"][i, j] == x[i, j]
                if j != jr:
                    n_other += 1
                    n_taken += taken
    frac = n_taken / n_other
    if CR in (0.0, 1.0):
        assert frac == CR
    else:
        sigma = math.sqrt(CR * (1 - CR) / n_other)
        assert abs(frac - CR) <= 5 * sigma, (frac, CR, sigma)


def test_taken_components_are_the_repaired_mutant():
    # F = 1.5 on populations spread over the ranges: many mutants leave them
    rng = np.random.default_rng(3)
    pop, F = 64, 1.5
    below = above = wrapped = 0
    for bounds in (BOUNDS5, np.vstack([BOUNDS5[:1], [[-1.0, 1.0]], BOUNDS5[2:]])):
        full_circle = bounds[1, 1] - bounds[1, 0] >= 2 * math.pi * (1 - 1e-12)
        for g in range(1, 21):
            x = _population(rng, pop, bounds)
            t = oracle.de_trials(5, 0, g, x, rng.random(pop), bounds, F, 1.0)
            v = _rand1_mutants(x, t["r"].astype(np.int64), F)
            assert np.all(t["take"] == 31)
            for i in range(pop):
                for j in range(5):
                    lo, hi, parent, u = bounds[j, 0], bounds[j, 1], x[i, j], t["u"][i, j]
                    if j == 1 and full_circle:
                        turns = (u - v[i, j]) / (2 * math.pi)
                        assert abs(turns - round(turns)) < 1e-9
                        assert lo <= u < lo + 2 * math.pi
                        wrapped += round(turns) != 0
                    elif v[i, j] < lo:
                        assert u == (lo + parent) / 2.0, (j, v[i, j], u)
                        below += 1
                    elif v[i, j] > hi:
                        assert u == (hi + parent) / 2.0, (j, v[i, j], u)
                        above += 1
                    else:
                        assert u == v[i, j]
    assert below > 100 and above > 100 and wrapped > 20


def test_either_or_coin_is_fair_and_applies_no_crossover():
    rng = np.random.default_rng(9)
    pop, F = 128, 0.6
    K = (F + 1.0) * 0.5
    n, heads = 0, 0
    for g in range(1, 61):
        x = _narrow_phase(_population(rng, pop, BOUNDS5))
        t = oracle.de_trials(21, 1, g, x, rng.random(pop), WIDE, F, 0.2, strategy="eitheror")
        assert np.all(t["take"] == 31)
        r = t["r"].astype(np.int64)
        a, b, c = x[r[:, 0]], x[r[:, 1]], x[r[:, 2]]
        three = t["three_point"]
        want = np.where(three[:, None], a + K * ((b + c) - 2.0 * a), a + F * (b - c))
        assert np.array_equal(t["u"], want)
        n += pop
        heads += int(three.sum())
    sigma = math.sqrt(0.25 / n)
    assert abs(heads / n - 0.5) <= 5 * sigma


def test_best_jitter_factor_in_range_and_base_is_lowest_index_minimum():
    rng = np.random.default_rng(13)
    pop, F = 64, 0.7
    factors = []
    for g in range(1, 31):
        x = _narrow_phase(_population(rng, pop, BOUNDS5))
        fx = rng.random(pop) + 1.0
        lo_idx = sorted(rng.choice(pop, 3, replace=False))
        fx[lo_idx] = 0.25  # a three-way tie: the lowest index is the base
        t = oracle.de_trials(8, 2, g, x, fx, WIDE, F, 1.0, strategy="best1jitter")
        assert t["best"] == lo_idx[0]
        r = t["r"].astype(np.int64)
        d = x[r[:, 1]] - x[r[:, 2]]
        ok = np.abs(d) > 1e-3
        fj = (t["u"] - x[lo_idx[0]])[ok] / d[ok]
        factors.append(fj)
    fj = np.concatenate(factors)
    assert np.all(fj >= F - 1e-9) and np.all(fj < F + 1e-4 + 1e-9)
    u = (fj - F) / 1e-4
    assert abs(np.mean(u) - 0.5) < 0.02  # the jitter is uniform over its width


def _restated_generation(seed, block_id, g, x, fx, bounds, F, CR, strategy):
    """One generation from the definitions: Philox words (counter (group,
    individual, generation, block), key = seed), indices drawn without
    replacement from a list, jrand and the crossover test on raw words, the
    strategy's mutant, and the repair."""
    pop, dim = x.shape
    key = [seed & 0xFFFFFFFF, seed >> 32]

    def words(grp, i):
        return [int(v) for v in oracle.philox4x32_10([grp, i, g, block_id], key)]

    best = min(range(pop), key=lambda i: (fx[i], i))
    thr = int(CR * TWO32)
    u = x.copy()
    for i in range(pop):
        w = words(0, i) + words(1, i) + words(2, i) + words(3, i)
        remaining = [j for j in range(pop) if j != i]
        r = []
        for d in range(3):
            r.append(remaining.pop((w[d] * len(remaining)) >> 32))
        jrand = (w[3] * dim) >> 32
        three = strategy == "eitheror" and w[9] >= 1 << 31
        for j in range(dim):
            a, b, c = x[r[0], j], x[r[1], j], x[r[2], j]
            take = j == jrand or CR >= 1.0 or w[4 + j] < thr
            if strategy == "best1jitter":
                jw = w[9 + j] if j < 3 else w[12 + j - 3]
                v = x[best, j] + (F + 1e-4 * (jw / TWO32)) * (b - c)
            elif strategy == "eitheror":
                v = a + ((F + 1.0) / 2.0) * ((b + c) - 2.0 * a) if three else a + F * (b - c)
                take = True
            else:
                v = a + F * (b - c)
            if not take:
                continue
            lo, hi = bounds[j]
            if j == 1 and hi - lo >= 2 * math.pi * (1 - 1e-12):
                v = v - math.floor((v - lo) / (2 * math.pi)) * (2 * math.pi)
            elif v < lo:
                v = (lo + x[i, j]) / 2.0
            elif v > hi:
                v = (hi + x[i, j]) / 2.0
            u[i, j] = v
    return u


@pytest.mark.parametrize("strategy", ["rand1bin", "best1jitter", "eitheror"])
@pytest.mark.parametrize("pop,dim", [(4, 5), (17, 5), (33, 7)])
def test_generation_matches_restatement_bit_for_bit(strategy, pop, dim):
    rng = np.random.default_rng(pop * 10 + dim)
    bounds = np.vstack([BOUNDS5, [[-0.05, 0.05], [-1e-3, 1e-3]]])[:dim]
    for g, F, CR, seed in ((1, 0.7, 0.9, 0), (5, 1.4, 0.5, (7 << 32) | 3), (200, 0.3, 0.1, 12345)):
        x = _population(rng, pop, bounds)
        fx = rng.random(pop)
        got = oracle.de_trials(seed, 6, g, x, fx, bounds, F, CR, strategy=strategy)["u"]
        want = _restated_generation(seed, 6, g, x, fx, bounds, F, CR, strategy)
        assert np.array_equal(got, want), (strategy, g)


def test_de_loop_uses_the_pinned_generation():
    # the DE's first generation after the initial population equals de_trials
    # on that population (the loop calls the same step), selection then keeps
    # the trial when its SSE is at or below the parent's
    s = np.random.default_rng(0).normal(0, 1, 300)
    fs, t0 = 100.0, -1.495
    b = BOUNDS5
    p0, f0v, pop0, fit0 = oracle.de_solve(s, fs, t0, b, 8, 0, 0.7, 0.9, 4, block_id=2, return_population=True)
    p1, f1v, pop1, fit1 = oracle.de_solve(s, fs, t0, b, 8, 1, 0.7, 0.9, 4, block_id=2, return_population=True)
    t = oracle.de_trials(4, 2, 1, pop0, fit0, b, 0.7, 0.9)
    fu = oracle.sse_many(s, fs, t0, t["u"])
    keep = fu <= fit0
    assert np.array_equal(pop1, np.where(keep[:, None], t["u"], pop0))
    assert np.array_equal(fit1, np.where(keep, fu, fit0))
