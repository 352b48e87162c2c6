"""GPU parity of the FFT seed of the first block's ranges (Sec. 3.1.1,
pt_seed_bounds) against the oracle's seed.

The three pieces' FFTs run in FP32 on the GPU and in FP64 (numpy) in the
oracle: the peak bins agree (or, at a near-tie, the GPU's bin carries the
oracle's maximum power within 1e-5), the refined offsets within 1e-4 bins,
and the estimates and ranges accordingly. Seeded ranges contain the
sign-normalised truth, and a DE fit inside them reaches the truth's basin.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    c = pt.Context(0)
    yield c
    c.close()


def _blocks():
    out = [synth.single4096(s) for s in range(3)]
    out += [synth.paper400k(s, n=n) for s, n in ((0, 400_000), (1, 100_003), (2, 33_333))]
    out += [synth.paper400k(3, n=50_000, storage=synth.I8), synth.perigee400k(1, n=80_000)]
    # the shortest blocks: pieces of 16, 16 and 32 samples
    out += [synth.single4096(s, n=n) for s, n in ((4, 64), (5, 127), (6, 255))]
    return out


@pytest.mark.parametrize("i", range(11))
def test_seed_matches_oracle(ctx, i):
    blk = _blocks()[i]
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    g = ctx.seed_bounds()
    o = oracle.seed_bounds(blk.values(), blk.fs, blk.t0)
    Np = o["piece_len"]
    assert g["piece_len"] == Np
    x = blk.values()
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(Np) / Np)
    for k, (s, kk, delta, _) in enumerate(o["pieces"]):
        if g["peak_bin"][k] != kk:
            P = np.abs(np.fft.rfft(w * x[s:s + Np])) ** 2
            assert P[g["peak_bin"][k]] >= P[kk] * (1 - 1e-5)
            continue
        assert abs(g["peak_delta"][k] - delta) < 1e-4
    bin_hz = blk.fs / Np
    assert abs(g["f0"] - o["f0"]) < 2e-4 * bin_hz + 1e-4 * abs(o["f1"] * o["piece_times"][1])
    assert abs(g["f1"] - o["f1"]) < 2e-4 * bin_hz / (2 * Np / blk.fs)
    assert g["A"] == pytest.approx(o["A"], rel=1e-4)
    np.testing.assert_allclose(g["bounds"], o["bounds"], rtol=1e-4, atol=1e-3 * bin_hz)


def test_seed_on_bin_tone_and_errors(ctx):
    import paper_1906_10598_b300 as pt
    fs, n = 1000.0, 4096
    t0 = synth.centred_t0(n, fs)
    Np = 1024
    x = 1.3 * np.cos(0.4 + 2 * np.pi * (37 * fs / Np) * (t0 + np.arange(n) / fs))
    ctx.load_block(x, fs, t0)
    g = ctx.seed_bounds()
    assert g["peak_bin"] == [37, 37, 37] and max(abs(d) for d in g["peak_delta"]) < 1e-5
    assert g["f0"] == pytest.approx(37 * fs / Np, rel=1e-7) and g["A"] == pytest.approx(1.3, rel=1e-5)
    g2 = ctx.seed_bounds(0.05, 256)
    assert g2["piece_len"] == 256 and g2["bounds"][2, 1] - g2["bounds"][2, 0] == pytest.approx(0.1 * g2["f0"])
    for args in ((0.0, 0), (1.5, 0), (0.1, 100), (0.1, 8)):
        with pytest.raises(pt.PhaseTrackError):
            ctx.seed_bounds(*args)
    ctx.load_block(np.zeros(40), fs, 0.0)
    with pytest.raises(pt.PhaseTrackError):
        ctx.seed_bounds()


def test_seeded_fit_reaches_the_truth(ctx):
    # single4096-shaped blocks (4 s at 1 kHz): DE inside the paper's +-10 % ranges
    import paper_1906_10598_b300 as pt
    for seed in range(3):
        blk = synth.single4096(seed)
        ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
        b = ctx.seed_bounds()["bounds"][:5]
        p, f = ctx.de_solve(b, 64, 1250, 0.7, 0.9, 5, pt.TIER_F64)
        tr = blk.truth.copy()
        if tr[2] < 0:
            tr[1:5] = -tr[1:5]
        assert abs(p[2] - tr[2]) < 0.01 and abs(math.remainder(p[1] - tr[1], 2 * math.pi)) < 0.05
        assert f <= oracle.sse(blk.values(), blk.fs, blk.t0, blk.truth) * (1 + 1e-6)
