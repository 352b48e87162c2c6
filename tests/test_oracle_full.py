"""Pins of the oracle's full model (CPU): Eq. 2-2-2 with the amplitude slope c5
and the Taylor phase of Eq. 2-2-1 at order n = 4 (Sec. 3.2), parameters
theta = (A, phi0, f0, f1, f2, A1, f3), and the DE over its 7 parameters.

Each pin comes from outside the oracle's own formula:
* finite differences of the phase: for a quartic, the 4th forward difference
  is f3 h^4 and the 3rd is f2 h^3 + (3/2) f3 h^4 (a dropped /24, a wrong power
  or a swapped index fails);
* SSE closed forms on a zero signal at quarter/sixteenth-cycle sample phases,
  where the phase mod 1 follows from integer arithmetic and cos^2 takes the
  exact values cos^2(k pi / 8);
* the noise-energy identity at the truth of a synthetic block;
* reduction to the 5-parameter model when A1 = f3 = 0 (bit for bit);
* the DE over 7 parameters: sphere and Rosenbrock known minima, a noise-free
  full-model block fitted to SSE ~ 0 at the truth, and a parameter held fixed
  by equal bounds.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def test_full_phase_finite_differences():
    rng = np.random.default_rng(1)
    for _ in range(20):
        th = np.array([1.0, 0.0, rng.uniform(-50, 50), rng.uniform(-5, 5), rng.uniform(-2, 2), 0.0,
                       rng.uniform(-3, 3)])
        h = 0.5
        t0 = rng.uniform(-1, 1)
        p = [oracle.phase_cycles_full(th, t0 + k * h) for k in range(5)]
        d4 = p[4] - 4 * p[3] + 6 * p[2] - 4 * p[1] + p[0]
        assert d4 == pytest.approx(th[6] * h ** 4, abs=1e-11)
        # third difference at t0 = 0 (expansion point): f2 h^3 + 3/2 f3 h^4
        q = [oracle.phase_cycles_full(th, k * h) for k in range(4)]
        d3 = q[3] - 3 * q[2] + 3 * q[1] - q[0]
        assert d3 == pytest.approx(th[4] * h ** 3 + 1.5 * th[6] * h ** 4, abs=1e-11)
        # phi0 enters as phi0 / (2 pi)
        th2 = th.copy()
        th2[1] = 1.0
        assert oracle.phase_cycles_full(th2, 0.3) - oracle.phase_cycles_full(th, 0.3) == pytest.approx(
            1.0 / (2 * math.pi), abs=1e-13)


def test_full_amplitude_slope_closed_form():
    # f0 = fs/4 and t_i = i / fs: the phase is i/4 cycles, cos^2 = 1 at even i,
    # ~0 at odd i. A zero signal leaves SSE = sum_{k<K} (A + A1 (2k)/fs)^2.
    fs, n = 4.0, 1001
    K = (n + 1) // 2
    for A, A1 in ((1.0, 0.0), (1.0, 0.25), (2.0, -0.125), (0.5, 3.0)):
        th = np.array([A, 0.0, fs / 4, 0.0, 0.0, A1, 0.0])
        got = oracle.sse_full(np.zeros(n), fs, 0.0, th)
        a1 = 2 * A1 / fs  # amplitude step per even sample
        want = K * A * A + A * a1 * K * (K - 1) + a1 * a1 * (K - 1) * K * (2 * K - 1) / 6
        assert got == pytest.approx(want, rel=1e-12)
        # A(t) is A + A1 t, not A (1 + A1 t) or A - A1 t
        assert oracle.model_full(th, 8.0) == pytest.approx(A + A1 * 8.0, rel=1e-13)


_COS2 = [math.cos(k * math.pi / 8) ** 2 for k in range(16)]


@pytest.mark.parametrize("f3_sign", [1, -1])
def test_full_quartic_term_closed_form(f3_sign):
    # fs = 1, t_i = i, f0 = 1/8, f3 = 24/16 * sign: the phase is (2 i + sign i^4)/16
    # cycles. Reduce that integer mod 16 and use cos^2(2 pi k / 16) = cos^2(k pi / 8).
    n = 64
    th = np.array([1.5, 0.0, 1.0 / 8, 0.0, 0.0, 0.0, f3_sign * 1.5])
    got = oracle.sse_full(np.zeros(n), 1.0, 0.0, th)
    want = sum(1.5 ** 2 * _COS2[(2 * i + f3_sign * i ** 4) % 16] for i in range(n))
    assert got == pytest.approx(want, rel=1e-9)
    # per sample the model is 1.5 cos(k pi / 8), k = (2 i + sign i^4) mod 16;
    # at i = 1 the two signs give cos(3 pi / 8) and cos(pi / 8)
    for i in range(n):
        k = (2 * i + f3_sign * i ** 4) % 16
        assert oracle.model_full(th, float(i)) == pytest.approx(1.5 * math.cos(k * math.pi / 8), abs=1e-8)


def test_full_reduces_to_cubic_model_bitwise():
    blk = synth.single4096(2)
    rng = np.random.default_rng(3)
    x = blk.values()
    for _ in range(10):
        th5 = np.array([rng.uniform(0.5, 2), rng.uniform(-3, 3), rng.uniform(-100, 100), rng.uniform(-1, 1),
                        rng.uniform(-0.1, 0.1)])
        th7 = np.concatenate([th5, [0.0, 0.0]])
        assert oracle.sse_full(x, blk.fs, blk.t0, th7) == oracle.sse(x, blk.fs, blk.t0, th5)
        for t in (-1.3, 0.0, 0.7):
            assert oracle.model_full(th7, t) == oracle.model(th5, t)
    many = oracle.sse_full_many(x, blk.fs, blk.t0, np.tile(np.concatenate([blk.truth, [0.0, 0.0]]), (3, 1)))
    assert np.all(many == oracle.sse(x, blk.fs, blk.t0, blk.truth))


@pytest.mark.parametrize("seed", [0, 1])
def test_full_noise_energy_identity(seed):
    blk = synth.perigee400k(seed, n=40_000, storage=synth.F64)
    e = float(np.sum(blk.noise ** 2))
    assert oracle.sse_full(blk.values(), blk.fs, blk.t0, blk.truth) == pytest.approx(e, rel=1e-9)
    # the noise-free signal: SSE ~ 0 at the truth, and each extra term is needed
    clean = blk.values() - blk.noise
    assert oracle.sse_full(clean, blk.fs, blk.t0, blk.truth) < 1e-20 * blk.n
    for j in (5, 6):
        th = blk.truth.copy()
        th[j] = 0.0
        assert oracle.sse_full(clean, blk.fs, blk.t0, th) > 1e-12


def test_de_dim7_textbook():
    b = np.tile([-5.0, 5.0], (7, 1))
    x, f = oracle.de_textbook_dim("sphere", b, 40, 600, 0.7, 0.9, 5)
    assert f < 1e-12 and np.all(np.abs(x) < 1e-5)
    b = np.tile([-2.0, 2.0], (7, 1))
    x, f = oracle.de_textbook_dim("rosenbrock", b, 70, 4000, 0.7, 0.9, 6)
    assert f < 1e-8 and np.all(np.abs(x - 1.0) < 1e-3)


def test_de_dim5_generalisation_keeps_draws():
    # the dimension-general DE reproduces the 5-parameter DE exactly
    b = np.tile([-2.0, 2.0], (5, 1))
    for which in ("sphere", "rosenbrock"):
        x1, f1 = oracle.de_textbook(which, b, 24, 150, 0.7, 0.9, 11)
        x2, f2 = oracle.de_textbook_dim(which, b, 24, 150, 0.7, 0.9, 11)
        assert np.array_equal(x1, x2) and f1 == f2


def _clean_full_block(n=3000, fs=1000.0):
    truth = np.array([1.2, 0.9, 37.0, 2.5, -0.8, 0.05, 3.0])
    t0 = synth.centred_t0(n, fs)
    x = synth.clean_tone_full(truth, n, fs, t0)
    T = n / fs
    bounds = np.array([[1.0, 1.4], [-math.pi, math.pi], [36.5, 37.3], [2.0, 3.2], [-2.0, 0.5],
                       [-0.2 * 1.4 / T, 0.2 * 1.4 / T], [1.0, 5.0]])
    return x, fs, t0, truth, bounds


def test_de_full_noise_free_reaches_truth():
    x, fs, t0, truth, bounds = _clean_full_block()
    p, f = oracle.de_solve_full(x, fs, t0, bounds, 48, 1500, 0.7, 0.9, 3)
    assert f < 1e-10 * len(x)
    assert abs(math.remainder(p[1] - truth[1], 2 * math.pi)) < 1e-5
    assert np.allclose(p[[0, 2, 3, 4, 5]], truth[[0, 2, 3, 4, 5]], rtol=0, atol=1e-4)
    assert abs(p[6] - truth[6]) < 1e-2


def test_de_full_fixed_parameter_by_equal_bounds():
    x, fs, t0, truth, bounds = _clean_full_block()
    b = bounds.copy()
    b[6] = (truth[6], truth[6])
    p, f, pop, fit = oracle.de_solve_full(x, fs, t0, b, 32, 300, 0.7, 0.9, 4, return_population=True)
    assert np.all(pop[:, 6] == truth[6])
    assert np.all(np.isfinite(fit))
    with pytest.raises(ValueError):
        oracle.de_solve_full(x, fs, t0, b[:5], 32, 10, 0.7, 0.9, 4)


@pytest.mark.parametrize("strategy", ["best1jitter", "eitheror"])
def test_de_dim7_strategies_known_minima(strategy):
    # the paper's strategies "3" and "6" over 7 parameters: the sphere's and
    # Rosenbrock's known minima, and the noise-free full-model block's truth
    b = np.tile([-5.0, 5.0], (7, 1))
    x, f = oracle.de_textbook_dim("sphere", b, 40, 600, 0.7, 0.9, 5, strategy=strategy)
    assert f < 1e-12 and np.all(np.abs(x) < 1e-5)
    b = np.tile([-2.0, 2.0], (7, 1))
    x, f = oracle.de_textbook_dim("rosenbrock", b, 70, 2000, 0.7, 0.9, 6, strategy=strategy)
    assert f < 1e-8 and np.all(np.abs(x - 1.0) < 1e-3)
    x, fs, t0, truth, bounds = _clean_full_block()
    p, f = oracle.de_solve_full(x, fs, t0, bounds, 48, 1500, 0.7, 0.9, 3, strategy=strategy)
    assert f < 1e-10 * len(x) and np.allclose(p[[0, 2, 3, 4, 5]], truth[[0, 2, 3, 4, 5]], rtol=0, atol=1e-4)
    # over 5 parameters the dimension-general DE is the 5-parameter one
    b5 = np.tile([-2.0, 2.0], (5, 1))
    a = oracle.de_textbook("rosenbrock", b5, 24, 150, 0.7, 0.9, 11, strategy=strategy)
    c = oracle.de_textbook_dim("rosenbrock", b5, 24, 150, 0.7, 0.9, 11, strategy=strategy)
    assert np.array_equal(a[0], c[0]) and a[1] == c[1]
