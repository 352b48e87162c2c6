"""Host-only block-to-block tracking helpers (no GPU): running-time range
setting (Sec. 3.1.1) and the continuity check (Eq. 3-1-2), checked against the
oracle's Eq. 3-1-1 observables (themselves pinned to Appendix 1) and against
synthetic streams whose true next-block coefficients are known."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def pt():
    from paper_1906_10598_b300 import build
    build.build()
    import paper_1906_10598_b300 as m
    return m


def _appendix_blocks():
    rows = [l.split() for l in open(__file__.replace("test_tracking.py", "golden/appendix1_mex.txt"))
            if l.strip() and not l.startswith("#")]
    return [np.array([float(v) for v in r[2:6]]) for r in rows if r[0] == "block"]


def _theta_from_c(c):
    # c0 = phi0, c1 = 2 pi f0, c2 = pi f1, c3 = pi f2 / 3; amplitude is irrelevant here
    return np.array([1.0, c[0], c[1] / (2 * np.pi), c[2] / np.pi, 3 * c[3] / np.pi])


def test_continuity_matches_oracle_on_appendix1(pt):
    blocks = _appendix_blocks()
    T = 2.0
    for a, b in zip(blocks, blocks[1:]):
        ok, dphi, dfreq = pt.continuity(_theta_from_c(a), T, _theta_from_c(b), T, 0.05, 0.5)
        want_phi = abs(np.angle(np.exp(1j * (oracle.c_phase(a, T / 2) - oracle.c_phase(b, -T / 2)))))
        want_f = abs(oracle.c_freq(a, T / 2) - oracle.c_freq(b, -T / 2))
        assert dphi == pytest.approx(want_phi, abs=1e-6)
        assert dfreq == pytest.approx(want_f, rel=1e-9, abs=1e-9)
        assert ok  # the paper's blocks are continuous within the ~50 mrad noise
    # a phase jump breaks continuity
    a, b = _theta_from_c(blocks[0]), _theta_from_c(blocks[1])
    b2 = b.copy()
    b2[1] += 0.3
    ok, dphi, _ = pt.continuity(a, T, b2, T, 0.05, 0.5)
    assert not ok and dphi > 0.2


def test_warm_bounds_contain_next_block_truth(pt):
    for spec in synth.make_streams(3):
        T = spec.block_s
        for k in range(3):
            tc = (k + 0.5) * T
            prev = synth.stream_taylor_truth(spec, tc)
            nxt = synth.stream_taylor_truth(spec, tc + T)
            b = pt.warm_bounds(prev, T, T)
            assert b[1, 0] == pytest.approx(-np.pi) and b[1, 1] == pytest.approx(np.pi)
            for j in (0, 2, 3, 4):
                assert b[j, 0] <= nxt[j] <= b[j, 1], (j, b[j], nxt[j])
            # the f0 range covers the frequency across the next block (Eq. 3-1-1)
            f_edges = [prev[2] + prev[3] * t + prev[4] * t * t / 2 for t in (T / 2, 3 * T / 2)]
            assert b[2, 0] <= min(f_edges) and b[2, 1] >= max(f_edges)


def test_warm_bounds_rejects_bad_input(pt):
    with pytest.raises(pt.PhaseTrackError):
        pt.warm_bounds([1, 0, 0, 0, np.nan], 1.0, 1.0)
    with pytest.raises(pt.PhaseTrackError):
        pt.warm_bounds([1, 0, 0, 0, 0], 1.0, 0.0)


def test_continuity_full_matches_oracle_quartic_phase(pt):
    rng = np.random.default_rng(4)
    for _ in range(20):
        a = np.array([1.0, rng.uniform(-3, 3), rng.uniform(-200, 200), rng.uniform(-5, 5), rng.uniform(-0.5, 0.5),
                      rng.uniform(-0.01, 0.01), rng.uniform(-0.01, 0.01)])
        b = a + rng.normal(0, [0, 0.01, 1e-3, 1e-3, 1e-4, 0, 1e-5])
        Ta, Tb = rng.uniform(1, 10), rng.uniform(1, 10)
        ok, dphi, dfreq = pt.continuity_full(a, Ta, b, Tb, 0.05, 0.5)
        pa = 2 * np.pi * oracle.phase_cycles_full(a, Ta / 2)
        pb = 2 * np.pi * oracle.phase_cycles_full(b, -Tb / 2)
        assert dphi == pytest.approx(abs(np.angle(np.exp(1j * (pa - pb)))), abs=1e-6)
        # frequency: the oracle's phase derivative by a central difference
        h = 1e-4
        fa = 2 * np.pi * (oracle.phase_cycles_full(a, Ta / 2 + h) - oracle.phase_cycles_full(a, Ta / 2 - h)) / (2 * h)
        fb = 2 * np.pi * (oracle.phase_cycles_full(b, -Tb / 2 + h) - oracle.phase_cycles_full(b, -Tb / 2 - h)) / (2 * h)
        assert dfreq == pytest.approx(abs(fa - fb), abs=1e-4)
        # with A1 = f3 = 0 it is the cubic check
        a5, b5 = a.copy(), b.copy()
        a5[5:] = 0.0
        b5[5:] = 0.0
        r7 = pt.continuity_full(a5, Ta, b5, Tb, 0.05, 0.5)
        r5 = pt.continuity(a5[:5], Ta, b5[:5], Tb, 0.05, 0.5)
        assert r7[0] == r5[0] and r7[1] == pytest.approx(r5[1], abs=1e-9) and r7[2] == pytest.approx(r5[2], rel=1e-12)


def test_warm_bounds_full_contain_next_block_truth(pt):
    specs = synth.make_streams(3) + [synth.perigee_stream(s) for s in range(3)]
    for spec in specs:
        T = spec.block_s
        a1 = (spec.A1 - 0.2 * spec.A / T, spec.A1 + 0.2 * spec.A / T)
        for k in range(4):
            tc = (k + 0.5) * T
            prev = synth.stream_taylor_truth_full(spec, tc)
            nxt = synth.stream_taylor_truth_full(spec, tc + T)
            b = pt.warm_bounds_full(prev, T, T, a1)
            assert b[1, 0] == pytest.approx(-np.pi) and b[1, 1] == pytest.approx(np.pi)
            for j in (0, 2, 3, 4, 5, 6):
                assert b[j, 0] <= nxt[j] <= b[j, 1], (spec.stream_id, k, j, b[j], nxt[j])
            assert tuple(b[5]) == a1
    with pytest.raises(pt.PhaseTrackError):
        pt.warm_bounds_full(np.full(7, np.nan), 1.0, 1.0)
    with pytest.raises(pt.PhaseTrackError):
        pt.warm_bounds_full(np.ones(7), 1.0, 1.0, (1.0, 0.0))
