"""Pins of the oracle's tracking session (oracle/track.py): Sec. 3.1.1
running-time ranges, the Eq. 3-1-2 continuity check, Sec. 3.1.4
enlarge-and-retry with abandonment, and Eq. 4-1-2 count intervals.

* Appendix 1 (the paper's printed MEX example): border phases and
  frequencies and the per-block total phase of its three fitted blocks, and
  their chaining into one count interval.
* Streams whose phase is an exact cubic: the next block's true coefficients
  are the extrapolated ones, so they sit at the centres of the running
  ranges; consecutive truths pass the continuity check with zero residual;
  the total phases of contiguous blocks add up to the stream's phase change.
* A scripted solver fixes each search's outcome, so the session's decisions
  (quality, attempts, widened ranges, Philox keys, abandonment, the gap
  extrapolation and the interval reset) are checked without any fit.
"""
import math

import numpy as np
import pytest

import synth
from oracle import track


def _appendix_rows():
    rows = [l.split() for l in open(__file__.replace("test_oracle_track.py", "golden/appendix1_mex.txt"))
            if l.strip() and not l.startswith("#")]
    blocks = [[float(v) for v in r[2:]] for r in rows if r[0] == "block"]
    borders = [[float(v) for v in r[2:]] for r in rows if r[0] == "border"]
    return blocks, borders


def _theta_from_c(c):
    # c0 = phi0, c1 = 2 pi f0, c2 = pi f1, c3 = pi f2 / 3, c4 = A, c5 = A1
    return np.array([c[4], c[0], c[1] / (2 * np.pi), c[2] / np.pi, 3 * c[3] / np.pi, c[5], 0.0])


def test_appendix1_borders_total_phase_and_interval():
    blocks, borders = _appendix_rows()
    T = 2.0
    fits = [_theta_from_c(b[:6]) for b in blocks]
    it = iter(fits)

    def solver(values, fs, t0, ranges, seed, block_id):
        return next(it), 1.0

    s = track.TrackSession(np.array([[0, 1e4], [-np.pi, np.pi], [0, 1e5], [-100, 100], [-10, 10],
                                     [-1e3, 1e3], [-1, 1]]), max_dphi=0.05, max_dfreq=0.5,
                           count_interval=3 * T, solver=solver)
    recs = [s.block(np.zeros(4), 2.0) for _ in fits]  # 4 samples at 2 Hz: T = 2 s
    for k, (b, r) in enumerate(zip(blocks, recs)):
        assert r["quality"] == 1 and r["attempts"] == 1
        # the printed total phase (c1 T + c3 T^3 / 4 at 3 decimals of each c)
        assert r["total_phase"] == pytest.approx(b[6], abs=2e-3)
        # border rows: left of block k is row 2k, right is row 2k + 1 (phase mod 2 pi, rad/s)
        left, right = borders[2 * k], borders[2 * k + 1]
        assert abs(math.remainder(r["phi_left"] - left[0], 2 * np.pi)) < 3e-3
        assert abs(math.remainder(r["phi_right"] - right[0], 2 * np.pi)) < 3e-3
        assert r["f_left"] == pytest.approx(left[1], abs=3e-3)
        assert r["f_right"] == pytest.approx(right[1], abs=3e-3)
        if k:
            # the paper's blocks are continuous within its noise (Eq. 3-1-2)
            assert r["dphi"] < 0.05 and r["dfreq"] < 0.5
    assert math.isnan(recs[0]["int_doppler"]) and math.isnan(recs[1]["int_doppler"])
    total = sum(b[6] for b in blocks)
    assert recs[2]["interval_phase"] == pytest.approx(total, abs=6e-3)
    assert recs[2]["int_doppler"] == pytest.approx(total / (3 * T), abs=1e-3)


class CubicStream:
    """Phase 2 pi (F0 t + F1 t^2/2 + F2 t^3/6) + P0 (stream time t), amplitude A."""

    def __init__(self, A=1.3, P0=0.4, F0=1234.5, F1=-3.25, F2=0.041):
        self.A, self.P0, self.F0, self.F1, self.F2 = A, P0, F0, F1, F2

    def phase(self, t):
        return self.P0 + 2 * np.pi * (self.F0 * t + self.F1 * t * t / 2 + self.F2 * t ** 3 / 6)

    def truth(self, tc):
        """The Taylor coefficients about tc (Eq. 2-2-3), exact for a cubic."""
        F0, F1, F2 = self.F0, self.F1, self.F2
        phi = math.remainder(self.phase(tc), 2 * np.pi)
        return np.array([self.A, phi, F0 + F1 * tc + F2 * tc * tc / 2, F1 + F2 * tc, F2])


def test_running_ranges_centre_on_the_extrapolated_truth():
    st = CubicStream()
    for T in (1.0, 2.0, 6.7):
        for gap_blocks in (0, 1, 3):
            prev = st.truth(0.5 * T)
            dt = T * (1 + gap_blocks)
            nxt = st.truth(0.5 * T + dt)
            r = track.running_ranges(prev, dt, T, 5)
            assert r[1, 0] == -np.pi and r[1, 1] == np.pi
            assert r[0] == pytest.approx([0.9 * st.A, 1.1 * st.A], rel=1e-15)
            for j in (2, 3, 4):
                assert r[j, 0] <= nxt[j] <= r[j, 1]
            # f2 about the previous value with the minimum half-width; f0 spans
            # the extrapolated frequency across the next block (at least 2/T either side)
            assert r[4] == pytest.approx([st.F2 - 24 / T ** 3, st.F2 + 24 / T ** 3], rel=1e-12)
            fl, fr = (st.truth(0.5 * T + dt + s * T / 2)[2] for s in (-1, 1))
            assert r[2, 0] == pytest.approx(min(fl, fr, nxt[2] - 2 / T), rel=1e-12)
            assert r[2, 1] == pytest.approx(max(fl, fr, nxt[2] + 2 / T), rel=1e-12)
            rates = [st.truth(0.5 * T + dt + s * T / 2)[3] for s in (-1, 1)]
            assert r[3, 0] == pytest.approx(min(*rates, nxt[3] - 4 / T ** 2), rel=1e-12)
            assert r[3, 1] == pytest.approx(max(*rates, nxt[3] + 4 / T ** 2), rel=1e-12)


def test_running_ranges_full_model_contain_next_truth():
    for spec in synth.make_streams(3) + [synth.perigee_stream(s) for s in range(3)]:
        T = spec.block_s
        a1 = (spec.A1 - 0.2 * spec.A / T, spec.A1 + 0.2 * spec.A / T)
        for k in range(4):
            prev = synth.stream_taylor_truth_full(spec, (k + 0.5) * T)
            nxt = synth.stream_taylor_truth_full(spec, (k + 1.5) * T)
            r = track.running_ranges(prev, T, T, 7, a1)
            for j in (0, 2, 3, 4, 5, 6):
                assert r[j, 0] <= nxt[j] <= r[j, 1], (spec.stream_id, k, j)
            assert tuple(r[5]) == a1
            assert r[6] == pytest.approx([prev[6] - 192 / T ** 4, prev[6] + 192 / T ** 4], rel=1e-12)


def test_continuity_of_consecutive_truths_and_of_a_phase_jump():
    st = CubicStream()
    T = 2.0
    a, b = st.truth(1.0), st.truth(3.0)
    dphi, dfreq = track.continuity(a, T, b, T)
    assert dphi < 1e-9 and dfreq < 1e-9
    b2 = b.copy()
    b2[1] += 0.25
    assert track.continuity(a, T, b2, T)[0] == pytest.approx(0.25, abs=1e-9)
    b3 = b.copy()
    b3[2] += 0.01  # 0.01 Hz at the border: 2 pi 0.01 rad/s
    assert track.continuity(a, T, b3, T)[1] == pytest.approx(2 * np.pi * 0.01, rel=1e-6)
    # phase compared mod 2 pi
    b4 = b.copy()
    b4[1] += 2 * np.pi
    assert track.continuity(a, T, b4, T)[0] < 1e-9
    # the frequency is the derivative of the phase (central difference)
    h = 1e-5
    for t in (-1.0, 0.3, 1.0):
        fd = (track.phase_rad(b, t + h) - track.phase_rad(b, t - h)) / (2 * h)
        assert track.freq_rad(b, t) == pytest.approx(fd, rel=1e-7)


def test_total_phases_of_contiguous_blocks_add_to_the_stream_phase_change():
    st = CubicStream()
    T = 2.5
    tot = sum(track.total_phase(st.truth((k + 0.5) * T), T) for k in range(4))
    assert tot == pytest.approx(st.phase(4 * T) - st.phase(0.0), rel=1e-13)
    # and each block's term is phi(T/2) - phi(-T/2) of its own fit (the even terms cancel)
    for k in range(4):
        p = st.truth((k + 0.5) * T)
        assert track.total_phase(p, T) == pytest.approx(track.phase_rad(p, T / 2) - track.phase_rad(p, -T / 2),
                                                        rel=1e-13)
    q = np.array([1.0, 0.1, 30.0, 2.0, 0.3, 0.01, 0.02])  # the full model's quartic term is even too
    assert track.total_phase(q, T) == pytest.approx(track.phase_rad(q, T / 2) - track.phase_rad(q, -T / 2),
                                                    rel=1e-12)


class Script:
    """A solver that returns the stream's truth for each block, shifted in
    phase by `bad[(block, search)]` radians (a failing search)."""

    def __init__(self, stream, T, bad):
        self.st, self.T, self.bad = stream, T, bad
        self.calls = []

    def __call__(self, values, fs, t0, ranges, seed, block_id):
        self.calls.append((block_id, seed, np.array(ranges)))
        search = sum(1 for c in self.calls if c[0] == block_id)
        p = self.st.truth((block_id + 0.5) * self.T)
        p[1] += self.bad.get((block_id, search), 0.0)
        return p, 1.0


def _session(script, **kw):
    T = script.T
    b = np.array([[0.5, 2.0], [-np.pi, np.pi], [1200, 1300], [-5, 5], [-0.1, 0.1]])
    args = dict(seed=40, max_dphi=0.1, max_dfreq=1.0, enlarge=2.5, max_attempts=3, count_interval=2 * T)
    args.update(kw)
    return track.TrackSession(b, solver=script, **args)


def test_retry_widens_ranges_and_advances_the_key():
    T, fs = 2.0, 2.0
    sc = Script(CubicStream(), T, {(1, 1): 1.0})
    s = _session(sc)
    r0 = s.block(np.zeros(4), fs)
    r1 = s.block(np.zeros(4), fs)
    assert (r0["quality"], r0["attempts"]) == (1, 1) and math.isnan(r0["dphi"])
    assert (r1["quality"], r1["attempts"]) == (2, 2)
    (b1, k1, g1), (b2, k2, g2) = sc.calls[1], sc.calls[2]
    assert (b1, b2) == (1, 1) and (k1, k2) == (40, 41)
    assert np.array_equal(g1, track.hold_fixed(track.running_ranges(r0["params"], T, T, 5), s.init))
    for j in (0, 2, 3, 4):
        assert (g2[j, 0] + g2[j, 1]) / 2 == pytest.approx((g1[j, 0] + g1[j, 1]) / 2, rel=1e-12)
        assert g2[j, 1] - g2[j, 0] == pytest.approx(2.5 * (g1[j, 1] - g1[j, 0]), rel=1e-12)
    assert np.array_equal(g2[1], g1[1])
    assert np.array_equal(r1["ranges"], g2)


def test_abandoned_block_breaks_adjacency_and_the_count_interval():
    T, fs = 2.0, 2.0
    st = CubicStream()
    sc = Script(st, T, {(2, 1): 1.0, (2, 2): 1.0, (2, 3): 1.0})
    s = _session(sc)
    recs = [s.block(np.zeros(4), fs) for _ in range(5)]
    q = [(r["quality"], r["attempts"]) for r in recs]
    assert q == [(1, 1), (1, 1), (0, 3), (1, 1), (1, 1)]
    assert math.isnan(recs[2]["total_phase"]) and math.isnan(recs[2]["int_doppler"])
    # the interval of blocks 0-1 completed at block 1; block 2 broke the next one
    assert recs[1]["interval_phase"] == pytest.approx(st.phase(2 * T) - st.phase(0.0), rel=1e-13)
    # block 3: no adjacent reference, accepted unchecked; its ranges are
    # extrapolated from block 1 across the abandoned block (dt = 2 T)
    assert math.isnan(recs[3]["dphi"])
    g3 = [c[2] for c in sc.calls if c[0] == 3][0]
    assert np.array_equal(g3, track.hold_fixed(track.running_ranges(recs[1]["params"], 2 * T, T, 5), s.init))
    # the interval restarted at block 3 and completes at block 4
    assert math.isnan(recs[3]["int_doppler"])
    assert recs[4]["interval_phase"] == pytest.approx(st.phase(5 * T) - st.phase(3 * T), rel=1e-12)
    assert recs[4]["dphi"] < 1e-9


def test_fixed_parameter_stays_fixed_and_amplitude_stays_positive():
    T, fs = 2.0, 2.0
    st = CubicStream()
    sc = Script(st, T, {(1, 1): 1.0, (1, 2): 1.0})
    b = np.array([[1.3, 1.3], [-np.pi, np.pi], [1200, 1300], [-5, 5], [-0.1, 0.1]])
    s = track.TrackSession(b, solver=sc, max_dphi=0.1, max_dfreq=1.0, enlarge=20.0, max_attempts=3)
    s.block(np.zeros(4), fs)
    r = s.block(np.zeros(4), fs)
    assert r["quality"] == 3
    for _, _, g in sc.calls:
        assert g[0, 0] == g[0, 1] == 1.3
    # with A free, a wide enlargement that would reach zero starts A at 1e-3 of its top
    w = track.widen(np.array([[0.9, 1.1], [-np.pi, np.pi], [0, 1], [0, 1], [0, 1]]), 20.0)
    assert w[0, 0] == pytest.approx(1e-3 * w[0, 1]) and w[0, 1] == pytest.approx(3.0)


def test_session_with_the_oracle_de_on_a_short_stream():
    # the oracle's own fits (no script): a clean 2-block stream is tracked
    # with both blocks accepted at the first search
    st = CubicStream(A=1.0, F0=40.0, F1=0.5, F2=0.0)
    fs, T = 400.0, 1.0
    n = int(fs * T)
    rng = np.random.default_rng(0)
    s = track.TrackSession(np.array([[0.8, 1.2], [-np.pi, np.pi], [39.0, 41.0], [0.0, 1.0], [-0.1, 0.1]]),
                           pop=24, gens=150, seed=2, max_dphi=0.2, max_dfreq=2.0)
    for k in range(2):
        t = k * T + np.arange(n) / fs
        x = st.A * np.cos(st.phase(t)) + rng.normal(0, 0.02, n)
        r = s.block(x, fs)
        tr = st.truth(k * T + (n - 1) / (2 * fs))
        assert r["quality"] == 1 and abs(r["params"][2] - tr[2]) < 0.01, (k, r["params"], tr)
