"""Pins of the oracle's FFT seed of the first block's ranges (Sec. 3.1.1, CPU).

* An on-bin tone: the periodic Hann window's spectrum of a tone at bin k has
  exactly three nonzero bins k-1, k, k+1 with equal outer magnitudes, so the
  refined offset is 0, the frequency is k fs / Np and the amplitude
  2 |X_k| / sum(w) is exact.
* An on-bin linear chirp: a windowed chirp symmetric about the window's
  centre has a spectrum symmetric about its centre frequency, so pieces whose
  centre frequencies fall on bins give those frequencies exactly, and the
  central difference gives the chirp rate exactly.
* Off-bin tones: the log-parabola refinement of the Hann spectrum stays within
  0.02 bins of the true frequency (its bias) and the corrected amplitude
  within 1 % (a sign error in the offset would cost up to a bin).
* A real tone cannot tell f0 from -f0: the seed takes the positive frequency,
  and its ranges contain the sign-normalised truth of the synthetic blocks.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _tone(n, fs, f, A=1.3, phi=0.4, f1=0.0, t_ref=0.0):
    t0 = synth.centred_t0(n, fs)
    t = t0 + np.arange(n) / fs
    return t0, A * np.cos(phi + 2 * np.pi * (f * (t - t_ref) + f1 * (t - t_ref) ** 2 / 2))


def test_piece_length_rule():
    assert oracle.seed_piece_len(4096) == 1024 and oracle.seed_piece_len(400_000) == 8192
    assert oracle.seed_piece_len(1000) == 128 and oracle.seed_piece_len(63) == 0


@pytest.mark.parametrize("k", [5, 37, 200])
def test_on_bin_tone_exact(k):
    fs, n = 1000.0, 4096
    Np = oracle.seed_piece_len(n)
    t0, x = _tone(n, fs, k * fs / Np)
    r = oracle.seed_bounds(x, fs, t0)
    for _, kk, delta, _ in r["pieces"]:
        assert kk == k and abs(delta) < 1e-12
    assert r["f0"] == pytest.approx(k * fs / Np, rel=1e-12)
    assert r["A"] == pytest.approx(1.3, rel=1e-12)
    assert abs(r["f1"]) < 1e-9


def test_on_bin_chirp_exact():
    # pieces centred (their sample Np/2) at times t_k; choose f(t) so that
    # f(t_k) = (k0 + (k - 1) m) fs / Np
    fs, n = 1000.0, 8192
    Np = oracle.seed_piece_len(n)
    t0 = synth.centred_t0(n, fs)
    tc = t0 + (n // 2) / fs  # the centre piece's time
    k0, m = 100, 3
    f1 = m * (fs / Np) / (Np / fs)
    t = t0 + np.arange(n) / fs
    x = 0.8 * np.cos(1.1 + 2 * np.pi * (k0 * fs / Np * (t - tc) + f1 * (t - tc) ** 2 / 2))
    r = oracle.seed_bounds(x, fs, t0)
    assert [p[1] for p in r["pieces"]] == [k0 - m, k0, k0 + m]
    assert r["f1"] == pytest.approx(f1, rel=1e-9)
    # f0 is the frequency at t = 0
    assert r["f0"] == pytest.approx(k0 * fs / Np - f1 * tc, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("d", [0.05, 0.2, 0.33, 0.45, 0.5, 0.7, 0.95])
def test_off_bin_tone_within_interpolation_bias(d):
    fs, n = 1000.0, 4096
    Np = oracle.seed_piece_len(n)
    f = (37 + d) * fs / Np
    t0, x = _tone(n, fs, f)
    r = oracle.seed_bounds(x, fs, t0)
    assert abs(r["f0"] - f) <= 0.02 * fs / Np
    assert r["A"] == pytest.approx(1.3, rel=1e-2)


def test_negative_frequency_gives_positive_seed():
    fs, n = 1000.0, 4096
    t0, x = _tone(n, fs, -123.4, f1=-2.0)
    r = oracle.seed_bounds(x, fs, t0)
    assert r["f0"] == pytest.approx(123.4, abs=0.05) and r["f1"] == pytest.approx(2.0, abs=0.2)


def test_ranges_contain_the_sign_normalised_truth():
    blocks = [synth.single4096(s) for s in range(4)] + [synth.paper400k(s, n=100_000) for s in range(4)]
    for blk in blocks:
        r = oracle.seed_bounds(blk.values(), blk.fs, blk.t0)
        tr = blk.truth.copy()
        if tr[2] < 0:  # (A, phi0, f0, f1, f2) and (A, -phi0, -f0, -f1, -f2) are the same signal
            tr[2:5] = -tr[2:5]
        b = r["bounds"]
        assert b.shape == (7, 2)
        for j in (2, 3, 4):
            assert b[j, 0] <= tr[j] <= b[j, 1], (j, b[j], tr[j])
        # the amplitude estimate is within the +-10 % range when the SNR allows it
        if blk.snr_db > 10:
            assert b[0, 0] <= tr[0] <= b[0, 1]
        assert b[1, 0] == -math.pi and b[1, 1] == math.pi


def test_too_short_block():
    with pytest.raises(ValueError):
        oracle.seed_bounds(np.zeros(40), 1000.0, 0.0)
