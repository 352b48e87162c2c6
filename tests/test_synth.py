"""Pins of the synthetic workloads' ground truth (CPU).

The serving workload's per-block truth is the cubic Taylor expansion of each
stream's continuous phase about the block centre (Eq. 2-2-3). Its truncation
error must respect the Lagrange bound of Eq. 3-2-2 at every sample of the
block, with n = 3:
    |R_3(t)| <= max |phi''''| |t - tc|^4 / 4!   (t - tc up to T/2).
A wrong sign or factor in any re-centred coefficient leaves a residual of
order |t - tc|, |t - tc|^2 or |t - tc|^3, far above that bound.
"""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("index", [0, 3, 17])
def test_stream_taylor_truth_within_lagrange_bound_eq_3_2_2(index):
    for spec in synth.make_streams(seed=5):
        n = int(round(spec.block_s * spec.fs))
        start = index * n
        tc = (start + (n - 1) / 2.0) / spec.fs
        tau = (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) / spec.fs
        truth = synth.stream_taylor_truth(spec, tc)
        # the stream's phase in cycles relative to the centre, and the cubic model
        p = synth.stream_phase_cycles(spec, tc + tau) - synth.stream_phase_cycles(spec, np.array([tc]))[0]
        model = truth[2] * tau + truth[3] * tau ** 2 / 2 + truth[4] * tau ** 3 / 6
        resid = np.abs(p - model)
        w = 2 * math.pi / spec.dop_p
        d4max = abs(spec.F3) + spec.dop_a * w ** 4  # |phi''''| in cycles/s^4, bound over the block
        bound = d4max * np.abs(tau) ** 4 / 24.0
        # cancellation in p (tens of thousands of cycles) limits the comparison to ~1e-9 cycles
        assert np.all(resid <= bound * (1 + 1e-9) + 1e-8), (spec.stream_id, float(np.max(resid - bound)))
        # and the border value matches Eq. 3-2-2's form |phi''''| T^4 / (2^4 4!)
        T = n / spec.fs
        assert resid.max() <= d4max * T ** 4 / (16 * 24) + 1e-8
        # the truth's phase is the stream's phase at the centre, wrapped to [-pi, pi)
        p0 = float(synth.stream_phase_cycles(spec, np.array([tc]))[0])
        assert math.isclose(math.remainder(truth[1] - 2 * math.pi * p0, 2 * math.pi), 0.0, abs_tol=1e-9)


def test_stream_taylor_truth_catches_a_wrong_coefficient():
    # the bound is tight enough to reject a perturbed linear or quadratic term
    spec = synth.make_streams(seed=5)[1]
    n = int(round(spec.block_s * spec.fs))
    tc = ((n - 1) / 2.0) / spec.fs
    tau = (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) / spec.fs
    truth = synth.stream_taylor_truth(spec, tc)
    p = synth.stream_phase_cycles(spec, tc + tau) - synth.stream_phase_cycles(spec, np.array([tc]))[0]
    w = 2 * math.pi / spec.dop_p
    bound = (abs(spec.F3) + spec.dop_a * w ** 4) * np.abs(tau) ** 4 / 24.0 + 1e-8
    for j, scale in ((2, 1e-6), (3, 1e-3), (4, 1e-2)):
        t2 = truth.copy()
        t2[j] += scale * (abs(t2[j]) + 1.0)
        model = t2[2] * tau + t2[3] * tau ** 2 / 2 + t2[4] * tau ** 3 / 6
        assert np.any(np.abs(p - model) > bound), j


@pytest.mark.parametrize("index", [0, 2, 5])
def test_stream_quartic_truth_within_lagrange_bound_eq_3_2_2(index):
    # the full model's truth (order n = 4) against Eq. 3-2-2 with n = 4:
    # |R_4(t)| <= max |phi^(5)| |t - tc|^5 / 5!, phi^(5) = a w^5 cos(w t) here
    specs = synth.make_streams(seed=5) + [synth.perigee_stream(1)]
    for spec in specs:
        n = int(round(spec.block_s * spec.fs))
        tc = (index * n + (n - 1) / 2.0) / spec.fs
        tau = (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) / spec.fs
        th = synth.stream_taylor_truth_full(spec, tc)
        p = synth.stream_phase_cycles(spec, tc + tau) - synth.stream_phase_cycles(spec, np.array([tc]))[0]
        model = th[2] * tau + th[3] * tau ** 2 / 2 + th[4] * tau ** 3 / 6 + th[6] * tau ** 4 / 24
        w = 2 * math.pi / spec.dop_p
        bound = spec.dop_a * w ** 5 * np.abs(tau) ** 5 / 120.0
        assert np.all(np.abs(p - model) <= bound * (1 + 1e-9) + 1e-8), spec.stream_id
        # the amplitude at the centre and its slope
        assert th[0] == pytest.approx(spec.A + spec.A1 * tc) and th[5] == spec.A1
        # dropping the quartic term leaves the order-4 remainder f3 tau^4 / 24 (up to the bound)
        if spec.F3 != 0.0 and spec.dop_a == 0.0:
            cubic = model - th[6] * tau ** 4 / 24
            assert np.max(np.abs(p - cubic)) == pytest.approx(abs(th[6]) * np.max(tau ** 4) / 24, rel=1e-6)
