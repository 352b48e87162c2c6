"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form,
an identity, a published known answer, a brute-force search, a textbook test
function or the paper's printed worked example (Appendix 1).
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
import synth

mpmath = pytest.importorskip("mpmath")


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al. SC'11) -- known answers


@pytest.mark.parametrize("ctr,key,want", [
    # Random123 known-answer vectors for philox4x32-10
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
])
def test_philox_random123_known_answers(ctr, key, want):
    assert [int(v) for v in oracle.philox4x32_10(ctr, key)] == want


def _curand_host_words(seed: int, nwords: int) -> np.ndarray:
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        pytest.skip("cuRAND host library not present")
    lib = ctypes.CDLL(path)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    buf = np.zeros(nwords, dtype=np.uint32)
    assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), nwords) == 0
    lib.curandDestroyGenerator(gen)
    return buf.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 1, 12345, 0xDEADBEEF, 0x0123456789ABCDEF])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host Philox4_32_10 generator (run as a library) emits, as its
    # k-th 4-word block, Philox of counter (k // 65536, 0, k % 65536, 0) keyed
    # by (seed lo, seed hi): 65536 subsequences in counter words 2-3, the
    # position inside a subsequence in word 0.
    ref = _curand_host_words(seed, 4 * (65536 + 4))
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in list(range(4)) + [65535, 65536, 65537, 65539]:
        ctr = [k // 65536, 0, k % 65536, 0]
        assert np.array_equal(oracle.philox4x32_10(ctr, key), ref[k]), k


# --------------------------------------------------------------------------
# Objective, Eq. 2-2-4 with the model of Eq. 2-2-2 (c5 = 0)


def _tone_sse_closed_form(n, fs, t0, a1, ph1, f1, a2, ph2, f2):
    """Sum_i (a1 cos(w1 t_i + ph1) - a2 cos(w2 t_i + ph2))^2 with t_i = t0 + i/fs,
    evaluated with the geometric-series (Dirichlet) closed form in 50-digit arithmetic."""
    mp = mpmath
    mp.mp.dps = 50

    def sum_cos(alpha, beta):  # sum_{i=0}^{n-1} cos(alpha + beta i)
        if abs(mp.sin(beta / 2)) < mp.mpf(10) ** -40:
            return n * mp.cos(alpha)
        return mp.sin(n * beta / 2) / mp.sin(beta / 2) * mp.cos(alpha + (n - 1) * beta / 2)

    w1 = 2 * mp.pi * mp.mpf(f1)
    w2 = 2 * mp.pi * mp.mpf(f2)
    t0m, fsm = mp.mpf(t0), mp.mpf(fs)
    a_1, b_1 = w1 * t0m + mp.mpf(ph1), w1 / fsm
    a_2, b_2 = w2 * t0m + mp.mpf(ph2), w2 / fsm
    s11 = mp.mpf(n) / 2 + sum_cos(2 * a_1, 2 * b_1) / 2
    s22 = mp.mpf(n) / 2 + sum_cos(2 * a_2, 2 * b_2) / 2
    s12 = (sum_cos(a_1 - a_2, b_1 - b_2) + sum_cos(a_1 + a_2, b_1 + b_2)) / 2
    return float(mp.mpf(a1) ** 2 * s11 + mp.mpf(a2) ** 2 * s22 - 2 * mp.mpf(a1) * mp.mpf(a2) * s12)


@pytest.mark.parametrize("case", range(6))
def test_sse_pure_tone_closed_form(case):
    rng = np.random.default_rng(100 + case)
    n = int(rng.integers(5, 3000))
    fs = float(rng.uniform(100, 20000))
    t0 = float(rng.uniform(-n / fs, n / fs))
    a1, ph1, f1 = rng.uniform(0.5, 2), rng.uniform(-3, 3), rng.uniform(-0.45, 0.45) * fs
    a2, ph2 = rng.uniform(0.5, 2), rng.uniform(-3, 3)
    f2 = f1 + (rng.uniform(-3, 3) * fs / n if case % 2 else 0.0)
    s = a1 * np.cos(2 * np.pi * f1 * (t0 + np.arange(n) / fs) + ph1)
    # the stored data carries FP64 rounding (~1e-16 per sample), far below the tolerance
    got = oracle.sse(s, fs, t0, [a2, ph2, f2, 0.0, 0.0])
    want = _tone_sse_closed_form(n, fs, t0, a1, ph1, f1, a2, ph2, f2)
    assert got == pytest.approx(want, rel=1e-9, abs=1e-9 * n)


def test_sse_at_truth_equals_noise_energy():
    # Sec. 2.2: at the true coefficients the chi-square converges to the noise power
    for seed in range(3):
        blk = synth.single4096(seed)
        got = oracle.sse(blk.values(), blk.fs, blk.t0, blk.truth)
        want = float(np.sum(blk.noise.astype(np.float64) ** 2))
        assert got == pytest.approx(want, rel=1e-10)


def test_sse_noiseless_truth_is_zero_and_quantised_truth_is_quantisation_energy():
    blk = synth.paper400k(3, n=20_000)
    clean = synth.clean_tone(blk.truth, blk.n, blk.fs, blk.t0)
    assert oracle.sse(clean, blk.fs, blk.t0, blk.truth) < 1e-18 * blk.n
    # quantised stored data: SSE(truth) = sum (stored value - clean)^2 exactly
    want = float(np.sum((blk.values() - clean) ** 2))
    assert oracle.sse(blk.values(), blk.fs, blk.t0, blk.truth) == pytest.approx(want, rel=1e-9)


def test_sse_invariances():
    blk = synth.paper400k(5, n=5_000)
    th = np.array(blk.truth) + np.array([0.1, 0.3, 0.05, 1e-3, 1e-5])
    base = oracle.sse(blk.values(), blk.fs, blk.t0, th)
    # phi0 -> phi0 + 2 pi
    assert oracle.sse(blk.values(), blk.fs, blk.t0, th + [0, 2 * np.pi, 0, 0, 0]) == pytest.approx(base, rel=1e-11)
    # cos is even: (A, phi0, f0, f1, f2) and (A, -phi0, -f0, -f1, -f2) give the same model
    mirror = np.array([th[0], -th[1], -th[2], -th[3], -th[4]])
    assert oracle.sse(blk.values(), blk.fs, blk.t0, mirror) == pytest.approx(base, rel=1e-11)
    # A -> -A with phi0 -> phi0 + pi
    flip = np.array([-th[0], th[1] + np.pi, th[2], th[3], th[4]])
    assert oracle.sse(blk.values(), blk.fs, blk.t0, flip) == pytest.approx(base, rel=1e-11)


def test_sse_time_origin_covariance():
    # Re-expanding the Taylor phase about a shifted origin (Eq. 2-2-1 at another
    # centre) and shifting t0 by the same amount leaves every model sample unchanged.
    rng = np.random.default_rng(9)
    blk = synth.paper400k(7, n=8_000)
    for _ in range(4):
        A, phi0, f0, f1, f2 = blk.truth + rng.normal(0, 1e-3, 5)
        tau = float(rng.uniform(-3, 3))
        p0 = phi0 / (2 * np.pi) - f0 * tau + f1 * tau ** 2 / 2 - f2 * tau ** 3 / 6
        th2 = [A, 2 * np.pi * p0, f0 - f1 * tau + f2 * tau ** 2 / 2, f1 - f2 * tau, f2]
        a = oracle.sse(blk.values(), blk.fs, blk.t0, [A, phi0, f0, f1, f2])
        b = oracle.sse(blk.values(), blk.fs, blk.t0 + tau, th2)
        assert b == pytest.approx(a, rel=1e-8)


def test_sse_many_matches_single_rows():
    blk = synth.single4096(2, n=1000)
    rng = np.random.default_rng(1)
    cands = blk.bounds[:, 0] + rng.random((17, 5)) * (blk.bounds[:, 1] - blk.bounds[:, 0])
    many = oracle.sse_many(blk.values(), blk.fs, blk.t0, cands, nthreads=3)
    for c, v in zip(cands, many):
        assert v == oracle.sse(blk.values(), blk.fs, blk.t0, c)


def test_sse_tiny_block_high_precision():
    # N <= 8: the long-double sum of FP64 residuals agrees with 40-digit arithmetic
    mp = mpmath
    mp.mp.dps = 40
    rng = np.random.default_rng(4)
    for n in range(1, 9):
        fs, t0 = 37.0, -0.31
        s = rng.normal(0, 1, n)
        th = [1.3, -2.0, 5.2, 0.7, -0.4]
        want = mp.mpf(0)
        for i in range(n):
            t = mp.mpf(t0) + mp.mpf(i) / mp.mpf(fs)
            ph = mp.mpf(th[1]) + 2 * mp.pi * (mp.mpf(th[2]) * t + mp.mpf(th[3]) * t ** 2 / 2 + mp.mpf(th[4]) * t ** 3 / 6)
            want += (mp.mpf(s[i]) - mp.mpf(th[0]) * mp.cos(ph)) ** 2
        assert oracle.sse(s, fs, t0, th) == pytest.approx(float(want), rel=1e-12, abs=1e-14)


# --------------------------------------------------------------------------
# Correlation objective (Eq. 2-2-5 with the constant-amplitude model, Eq. 2-2-6)


@pytest.mark.parametrize("case", range(4))
def test_cor_full_cycle_tone_closed_form(case):
    # s = A0 cos(2 pi f t + ph) over a whole number of cycles, with 2 f not a
    # multiple of fs: sum cos^2 = N/2, so cor at the truth with amplitude A is
    # A A0 N / 2 and F_cor = 1 / (atan(A A0 N / 2) + pi/2)
    rng = np.random.default_rng(300 + case)
    n = int(rng.integers(50, 4000))
    fs = float(rng.uniform(100, 20000))
    k = int(rng.integers(1, n // 3))
    f = k * fs / n
    t0 = 0.0
    a0, ph, a = rng.uniform(0.5, 2), rng.uniform(-3, 3), rng.uniform(0.1, 3)
    s = a0 * np.cos(2 * np.pi * f * np.arange(n) / fs + ph)
    th = [a, ph, f, 0.0, 0.0]
    want = a * a0 * n / 2
    assert oracle.cor(s, fs, t0, th) == pytest.approx(want, rel=1e-11, abs=1e-9)
    assert oracle.cor_objective(s, fs, t0, th) == pytest.approx(1.0 / (math.atan(want) + math.pi / 2), rel=1e-12)
    # a candidate j/T away in frequency is orthogonal: cor = 0, F_cor = 2/pi
    j = int(rng.integers(1, 5))
    off = [a, ph, f + j * fs / n, 0.0, 0.0]
    assert abs(oracle.cor(s, fs, t0, off)) < 1e-9 * n
    assert oracle.cor_objective(s, fs, t0, off) == pytest.approx(2 / math.pi, rel=1e-9)


def test_cor_phase_flip_identity_and_limit():
    # cos(x + pi) = -cos(x) gives cor(theta + pi) = -cor(theta), hence
    # 1/F(theta) + 1/F(theta + pi) = pi for any data; and F -> 1/pi as cor grows
    blk = synth.paper400k(5, n=4096)
    s = blk.values()
    rng = np.random.default_rng(1)
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    for _ in range(5):
        th = lo + rng.random(5) * (hi - lo)
        flip = th.copy()
        flip[1] += math.pi
        c1, c2 = oracle.cor(s, blk.fs, blk.t0, th), oracle.cor(s, blk.fs, blk.t0, flip)
        assert c2 == pytest.approx(-c1, rel=1e-9, abs=1e-9 * blk.n)
        f1 = oracle.cor_objective(s, blk.fs, blk.t0, th)
        f2 = oracle.cor_objective(s, blk.fs, blk.t0, flip)
        assert 1 / f1 + 1 / f2 == pytest.approx(math.pi, rel=1e-12)
    tr = np.array(blk.truth)
    vals = []
    for scale in (1.0, 10.0, 100.0):
        t = tr.copy()
        t[0] *= scale
        vals.append(oracle.cor_objective(s, blk.fs, blk.t0, t))
    assert all(v > 1 / math.pi for v in vals) and vals[0] > vals[1] > vals[2]
    assert vals[2] - 1 / math.pi < 1e-5


def test_cor_tiny_block_high_precision_and_many():
    mp = mpmath
    mp.mp.dps = 40
    rng = np.random.default_rng(6)
    for n in range(1, 9):
        fs, t0 = 37.0, -0.31
        s = rng.normal(0, 1, n)
        th = [1.3, -2.0, 5.2, 0.7, -0.4]
        want = mp.mpf(0)
        for i in range(n):
            t = mp.mpf(t0) + mp.mpf(i) / mp.mpf(fs)
            ph = mp.mpf(th[1]) + 2 * mp.pi * (mp.mpf(th[2]) * t + mp.mpf(th[3]) * t ** 2 / 2 + mp.mpf(th[4]) * t ** 3 / 6)
            want += mp.mpf(s[i]) * mp.mpf(th[0]) * mp.cos(ph)
        assert oracle.cor(s, fs, t0, th) == pytest.approx(float(want), rel=1e-12, abs=1e-14)
        assert oracle.cor_objective(s, fs, t0, th) == pytest.approx(float(1 / (mp.atan(want) + mp.pi / 2)), rel=1e-13)
    blk = synth.paper400k(7, n=1000)
    cands = blk.bounds[:, 0] + rng.random((9, 5)) * (blk.bounds[:, 1] - blk.bounds[:, 0])
    many = oracle.cor_objective_many(blk.values(), blk.fs, blk.t0, cands, nthreads=3)
    for c, v in zip(cands, many):
        assert v == oracle.cor_objective(blk.values(), blk.fs, blk.t0, c)


def test_de_on_cor_objective_finds_the_chi2_basin():
    # With A held constant (lo = hi), minimising F_cor maximises the
    # cross-correlation: on a tiny block it reaches the same (phi0, f0, f1)
    # basin as the chi-square fit, and no point of a dense grid beats it.
    rng = np.random.default_rng(0)
    fs, n = 100.0, 64
    t0 = synth.centred_t0(n, fs)
    truth = np.array([1.0, 0.7, 3.1, 0.4, 0.0])
    s = synth.clean_tone(truth, n, fs, t0) + rng.normal(0, 0.1, n)
    bounds = np.array([[1.0, 1.0], [-np.pi, np.pi], [2.9, 3.3], [-1.0, 1.5], [-0.5, 0.5]])
    x, f = oracle.de_solve(s, fs, t0, bounds, 40, 400, 0.7, 0.9, 5, objective="cor")
    assert x[0] == 1.0
    assert f == oracle.cor_objective(s, fs, t0, x)
    grid = [[1.0, ph, f0, f1, 0.0] for ph in np.linspace(-np.pi, np.pi, 41)
            for f0 in np.linspace(2.9, 3.3, 41) for f1 in np.linspace(-1.0, 1.5, 21)]
    gvals = oracle.cor_objective_many(s, fs, t0, np.array(grid))
    assert f <= gvals.min() + 1e-12
    xc, _ = oracle.de_solve(s, fs, t0, bounds, 40, 400, 0.7, 0.9, 5)
    assert abs(x[2] - xc[2]) < 0.02 and abs(np.angle(np.exp(1j * (x[1] - xc[1])))) < 0.2


# --------------------------------------------------------------------------
# Differential Evolution (Sec. 1.2, Table 3-1-1)


def test_de_textbook_sphere_converges():
    b = np.array([[-5.0, 5.0]] * 5)
    x, f = oracle.de_textbook("sphere", b, pop=30, gens=600, F=0.5, CR=0.9, seed=1)
    assert f < 1e-12
    assert np.all(np.abs(x) < 1e-6)


def test_de_textbook_rosenbrock_converges():
    b = np.array([[-2.0, 2.0]] * 5)
    x, f = oracle.de_textbook("rosenbrock", b, pop=40, gens=4000, F=0.7, CR=0.9, seed=3)
    assert f < 1e-6
    assert np.allclose(x, 1.0, atol=1e-2)


@pytest.mark.parametrize("strategy", ["rand1bin", "best1jitter", "eitheror"])
def test_de_strategies_converge_on_sphere(strategy):
    b = np.array([[-5.0, 5.0]] * 5)
    x, f = oracle.de_textbook("sphere", b, pop=30, gens=800, F=0.5, CR=0.9, seed=1, strategy=strategy)
    assert f < 1e-12 and np.all(np.abs(x) < 1e-6)


def _rosenbrock_grad(x):
    g = np.zeros_like(x)
    for j in range(len(x) - 1):
        a = x[j + 1] - x[j] ** 2
        g[j] += -400.0 * x[j] * a - 2.0 * (1.0 - x[j])
        g[j + 1] += 200.0 * a
    return g


def test_de_either_or_solves_rosenbrock():
    b = np.array([[-2.0, 2.0]] * 5)
    x, f = oracle.de_textbook("rosenbrock", b, pop=40, gens=8000, F=0.8, CR=0.9, seed=3, strategy="eitheror")
    assert f < 1e-12 and np.allclose(x, 1.0, atol=1e-6)


def test_de_best1_jitter_reaches_a_stationary_point():
    # the greedy best/1 settles on the 5-D Rosenbrock function's other local
    # minimum (x1 ~ -0.96); whichever minimum it reports, the gradient there
    # must vanish (an independent check of the search, not of its formula)
    b = np.array([[-2.0, 2.0]] * 5)
    x, f = oracle.de_textbook("rosenbrock", b, pop=40, gens=4000, F=0.5, CR=0.9, seed=0, strategy="best1jitter")
    assert np.linalg.norm(_rosenbrock_grad(x)) < 1e-4
    assert f < 1e-8 or 3.9 < f < 3.95


@pytest.mark.parametrize("strategy,objective", [("best1jitter", "chi2"), ("eitheror", "cor")])
def test_de_strategies_beat_brute_force_grid(strategy, objective):
    # the paper's pairings (Sec. 3.1.2): "3" with Eq. 2-2-4, "6" with Eq. 2-2-5
    rng = np.random.default_rng(0)
    fs, n = 100.0, 64
    t0 = synth.centred_t0(n, fs)
    truth = np.array([1.0, 0.7, 3.1, 0.4, 0.0])
    s = synth.clean_tone(truth, n, fs, t0) + rng.normal(0, 0.1, n)
    bounds = np.array([[0.8, 1.2], [-np.pi, np.pi], [2.9, 3.3], [-1.0, 1.5], [-0.5, 0.5]])
    if objective == "cor":
        bounds[0] = (1.0, 1.0)
    grid = np.array([[1.0, ph, f0, f1, 0.0] for ph in np.linspace(-np.pi, np.pi, 41)
                     for f0 in np.linspace(2.9, 3.3, 41) for f1 in np.linspace(-1.0, 1.5, 21)])
    gvals = (oracle.cor_objective_many if objective == "cor" else oracle.sse_many)(s, fs, t0, grid)
    x, f = oracle.de_solve(s, fs, t0, bounds, 40, 400, 0.7, 0.9, 5, objective=objective, strategy=strategy)
    assert f <= gvals.min() + 1e-9
    g = grid[int(np.argmin(gvals))]
    assert abs(x[2] - g[2]) < 0.02 and abs(np.angle(np.exp(1j * (x[1] - g[1])))) < 0.2


def test_de_prefix_monotone_and_in_bounds():
    # Counter-based draws make a run of G generations a prefix of a run of
    # G + k generations: the best objective can only improve.
    blk = synth.single4096(1, n=512)
    s = blk.values()
    best = []
    for g in (0, 5, 20, 60):
        x, f, pop, fit = oracle.de_solve(s, blk.fs, blk.t0, blk.bounds, 16, g, 0.7, 0.9, 42, return_population=True)
        best.append(f)
        assert np.all(pop >= blk.bounds[:, 0] - 1e-12) and np.all(pop <= blk.bounds[:, 1] + 1e-12)
        assert f == pytest.approx(fit.min())
        assert f == oracle.sse(s, blk.fs, blk.t0, x)
    assert all(b2 <= b1 for b1, b2 in zip(best, best[1:]))


def test_de_beats_brute_force_grid_on_tiny_block():
    # N = 64, narrow bounds: DE's optimum is no worse than the best point of a
    # dense grid over (phi0, f0, f1) with A and f2 at the truth.
    rng = np.random.default_rng(0)
    fs, n = 100.0, 64
    t0 = synth.centred_t0(n, fs)
    truth = np.array([1.0, 0.7, 3.1, 0.4, 0.0])
    s = synth.clean_tone(truth, n, fs, t0) + rng.normal(0, 0.1, n)
    bounds = np.array([[0.8, 1.2], [-np.pi, np.pi], [2.9, 3.3], [-1.0, 1.5], [-0.5, 0.5]])
    grid = []
    for ph in np.linspace(-np.pi, np.pi, 41):
        for f0 in np.linspace(2.9, 3.3, 41):
            for f1 in np.linspace(-1.0, 1.5, 21):
                grid.append([1.0, ph, f0, f1, 0.0])
    gvals = oracle.sse_many(s, fs, t0, np.array(grid))
    gmin = gvals.min()
    x, f = oracle.de_solve(s, fs, t0, bounds, 40, 400, 0.7, 0.9, 5)
    assert f <= gmin + 1e-9
    # and it lands in the grid optimum's basin
    g = np.array(grid[int(np.argmin(gvals))])
    assert abs(x[2] - g[2]) < 0.02 and abs(np.angle(np.exp(1j * (x[1] - g[1])))) < 0.2


@pytest.mark.slow
def test_de_errors_consistent_with_cramer_rao():
    # Estimation-theory check (not in the paper): on blocks where DE reaches the
    # global basin, errors of phi0/f0/f1 normalised by the exact-Fisher CRB are O(1).
    z = []
    for seed in range(12):
        blk = synth.single4096(seed)
        T = blk.T
        b = np.array(blk.bounds)
        rng = np.random.default_rng(seed)
        for j, hw in ((2, 2.0 / T), (3, 4.0 / T ** 2), (4, 24.0 / T ** 3)):
            c = blk.truth[j] + rng.uniform(-0.5, 0.5) * hw
            b[j] = (c - hw, c + hw)
        x, f = oracle.de_solve(blk.values(), blk.fs, blk.t0, b, 32, 300, 0.7, 0.9, seed)
        if f > oracle.sse(blk.values(), blk.fs, blk.t0, blk.truth) + 50 * blk.sigma ** 2:
            continue  # missed the global basin
        crb = oracle.crb(blk.truth, blk.n, blk.fs, blk.t0, blk.sigma)
        d = x - blk.truth
        d[1] = np.angle(np.exp(1j * d[1]))
        z.append(d[1:4] / crb[1:4])
    z = np.array(z)
    assert len(z) >= 8
    rms = np.sqrt(np.mean(z ** 2, axis=0))
    assert np.all(rms > 0.3) and np.all(rms < 2.5), rms
    assert np.max(np.abs(z)) < 5.0


# --------------------------------------------------------------------------
# Observables (Eq. 3-1-1, Eq. 4-1-2) against the paper's Appendix 1


def _appendix1():
    path = os.path.join(os.path.dirname(__file__), "golden", "appendix1_mex.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows.append((parts[0], [float(v) for v in parts[2:]]))
    return rows


def test_appendix1_total_phase_and_borders():
    rows = _appendix1()
    T = 2.0
    blocks = [(i, v) for i, (k, v) in enumerate(rows) if k == "block"]
    assert len(blocks) == 3
    for i, v in blocks:
        c = np.array(v[:4])
        # Eq. 4-1-2 for one block: phi(T/2) - phi(-T/2) = c1 T + c3 T^3 / 4
        assert oracle.c_total_phase(c, T) == pytest.approx(v[6], abs=4e-3)
        assert oracle.c_total_phase(c, T) == pytest.approx(c[1] * T + c[3] * T ** 3 / 4, rel=1e-14)
        left, right = rows[i - 1][1], rows[i + 1][1]
        # Eq. 3-1-1 border frequency and phase (mod 2 pi)
        assert oracle.c_freq(c, -T / 2) == pytest.approx(left[1], abs=4e-3)
        assert oracle.c_freq(c, T / 2) == pytest.approx(right[1], abs=4e-3)
        for got, want in ((oracle.c_phase(c, -T / 2), left[0]), (oracle.c_phase(c, T / 2), right[0])):
            d = abs(np.angle(np.exp(1j * (got % (2 * np.pi) - want))))
            assert d < 4e-3


def test_appendix1_continuity_eq_3_1_2():
    # adjacent blocks agree at their shared border within the ~50 mrad phase noise
    rows = _appendix1()
    T = 2.0
    blocks = [np.array(v[:4]) for k, v in rows if k == "block"]
    for a, b in zip(blocks, blocks[1:]):
        dphi = np.angle(np.exp(1j * (oracle.c_phase(a, T / 2) - oracle.c_phase(b, -T / 2))))
        assert abs(dphi) < 0.05
        assert abs(oracle.c_freq(a, T / 2) - oracle.c_freq(b, -T / 2)) < 0.5


def test_theta_to_c_and_total_phase_is_integral_of_frequency():
    th = [1.5, 0.4, 1234.5, -3.2, 0.04]
    c = oracle.theta_to_c(th)
    assert c[0] == 0.4 and c[4] == 1.5
    T = 7.0
    # total phase equals the integral of Eq. 3-1-1's F(t) over the block
    integ = mpmath.quad(lambda t: oracle.c_freq(c, float(t)), [-T / 2, T / 2])
    assert oracle.c_total_phase(c, T) == pytest.approx(float(integ), rel=1e-12)
    # and equals 2 pi (p(T/2) - p(-T/2)) of the cycles form
    want = 2 * np.pi * (oracle.phase_cycles(th, T / 2) - oracle.phase_cycles(th, -T / 2))
    assert oracle.c_total_phase(c, T) == pytest.approx(want, rel=1e-12)


def test_crb_matches_textbook_tone_formula():
    # For a pure tone (f1 = f2 = 0 fixed) the 3-parameter CRB of frequency is
    # sqrt(12 / ((2 pi)^2 SNR N (N^2 - 1))) * fs in Hz (Rife & Boorstyn 1974),
    # with SNR = A^2 / (2 sigma^2) and a centred time origin.
    n, fs, A, sigma = 2001, 1000.0, 1.0, 0.1
    t0 = synth.centred_t0(n, fs)
    t = t0 + np.arange(n) / fs
    ph = 0.3 + 2 * np.pi * 50.0 * t
    g = np.stack([np.cos(ph), -A * np.sin(ph), -A * np.sin(ph) * 2 * np.pi * t])
    crb3 = np.sqrt(np.diag(np.linalg.inv(g @ g.T / sigma ** 2)))
    snr = A * A / (2 * sigma * sigma)
    want = math.sqrt(12.0 / ((2 * math.pi) ** 2 * snr * n * (n * n - 1))) * fs
    assert crb3[2] == pytest.approx(want, rel=2e-3)
    # the oracle's 5-parameter CRB is never below the 3-parameter one
    assert oracle.crb([A, 0.3, 50.0, 0.0, 0.0], n, fs, t0, sigma)[2] >= crb3[2] * (1 - 1e-9)
