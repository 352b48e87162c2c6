"""GPU parity of the chi-square objective (Eq. 2-2-4) against the FP64 oracle.

Tolerances:
* default tier (FP64-anchored phase, FP32 cosine/residuals): |dSSE| <= 1e-6 SSE
  on noisy blocks (the bound the design targets); on blocks of a few samples
  (or a quiet ragged block) plus the propagation of the per-sample residual
  error, 2 sqrt(n SSE) dr + n dr^2 with dr = 2e-6 (smax + |A|), which
  dominates when the SSE is small (residual_term_bound);
* all-FP64 tier: 1e-9 relative (FP64 Horner in seconds vs the oracle's direct
  sum; CUDA cospi vs libm cos);
* double-float tier: 1e-5 relative; naive FP32 is reported, not bounded.
"""
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


def _candidates(blk, rng, nrand=12):
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    rows = [lo + rng.random(5) * (hi - lo) for _ in range(nrand)]
    tr = np.array(blk.truth, dtype=np.float64)
    rows.append(tr.copy())
    crb = oracle.crb(tr, blk.n, blk.fs, blk.t0, blk.sigma)
    for j in range(5):
        for sgn in (-1.0, 1.0):
            r = tr.copy()
            r[j] += sgn * crb[j]
            rows.append(r)
    far = tr.copy()
    far[2] += 37.0
    rows.append(far)
    amp = tr.copy()
    amp[0] *= 1.5
    rows.append(amp)
    return np.array(rows)


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


@pytest.mark.parametrize("storage", ["i16", "i8", "f16", "f32", "f64"])
def test_default_tier_matches_oracle(ctx, storage):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(11, n=20_000 + 77, storage=synth.STORAGE_NAMES[storage])
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    cands = _candidates(blk, np.random.default_rng(3))
    got = ctx.objective(cands, pt.TIER_F64)
    want = oracle.sse_many(blk.values(), blk.fs, blk.t0, cands)
    assert np.max(_rel(got, want)) <= 1e-6, _rel(got, want)


def test_plain_and_df32_tiers_match_oracle(ctx):
    import paper_1906_10598_b300 as pt
    blk = synth.single4096(4)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    cands = _candidates(blk, np.random.default_rng(5))
    want = oracle.sse_many(blk.values(), blk.fs, blk.t0, cands)
    plain = ctx.objective(cands, pt.TIER_PLAIN)
    assert np.max(_rel(plain, want)) <= 1e-9
    df = ctx.objective(cands, pt.TIER_DF32)
    assert np.max(_rel(df, want)) <= 1e-5
    f32 = ctx.objective(cands, pt.TIER_F32)
    assert np.all(np.isfinite(f32))


def test_default_tier_long_block_high_phase(ctx):
    # 40 s block at 10 kHz with f0 near 2 kHz: the phase reaches ~4e4 cycles
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(2)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    cands = _candidates(blk, np.random.default_rng(8), nrand=4)
    got = ctx.objective(cands, pt.TIER_F64)
    want = oracle.sse_many(blk.values(), blk.fs, blk.t0, cands)
    assert np.max(_rel(got, want)) <= 1e-6


def residual_term_bound(want, n, smax, amax):
    """|dSSE| allowed for the default tier: 1e-6 relative plus the propagation
    of a per-sample residual error |e_i| <= dr = 2e-6 (smax + |A|) (SFU cosine
    ~4e-7 |A|, FP32 phase walk ~1e-6 rad |A|, FP32 roundings of s and A, a
    factor 2 of margin): sum 2 r_i e_i + e_i^2 <= 2 sqrt(n SSE) dr + n dr^2
    by Cauchy-Schwarz. It dominates when a few samples leave a small SSE."""
    dr = 2e-6 * (smax + amax)
    return 1e-6 * want + 2.0 * np.sqrt(n * want) * dr + n * dr * dr


@pytest.mark.parametrize("n", [1, 7, 255, 256, 257, 513, 4099])
def test_ragged_and_tiny_blocks(ctx, n):
    import paper_1906_10598_b300 as pt
    fs = 1000.0
    t0 = synth.centred_t0(n, fs)
    truth = np.array([1.2, 0.4, 31.0, 0.3, 0.01])
    cands = np.array([truth, truth + [0.1, 0.2, 0.5, 0.1, 0.0], [0.7, -2.0, 12.0, -0.2, 0.0]])
    for sigma in (0.05, 0.3):
        rng = np.random.default_rng(n + int(sigma * 100))
        s = synth.clean_tone(truth, n, fs, t0) + rng.normal(0, sigma, n)
        ctx.load_block(s, fs, t0)
        want = oracle.sse_many(s, fs, t0, cands)
        got = ctx.objective(cands, pt.TIER_F64)
        bound = residual_term_bound(want, n, np.max(np.abs(s)), np.max(np.abs(cands[:, 0])))
        assert np.all(np.abs(got - want) <= bound), (sigma, np.abs(got - want), bound)
        if sigma == 0.3 and n >= 255:
            # noisy blocks of a tile or more: the 1e-6 relative bound alone
            assert np.max(_rel(got, want)) <= 1e-6, (sigma, _rel(got, want))
        plain = ctx.objective(cands, pt.TIER_PLAIN)
        assert np.max(_rel(plain, want)) <= 1e-9, _rel(plain, want)


def test_result_independent_of_batch_shape(ctx):
    # fixed-point accumulation: a candidate's SSE is bit-identical whatever
    # else is in the batch and however the launch is shaped
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(6, n=50_000)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    rng = np.random.default_rng(0)
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    cands = lo + rng.random((300, 5)) * (hi - lo)
    full = ctx.objective(cands, pt.TIER_F64)
    for k in (1, 3, 9, 129):
        part = ctx.objective(cands[:k].copy(), pt.TIER_F64)
        assert np.array_equal(part, full[:k])
    again = ctx.objective(cands, pt.TIER_F64)
    assert np.array_equal(again, full)


def test_whole_wave_grid_on_the_paper_block(ctx):
    # The 400K block against 4096 candidates is the one launch whose grid
    # takes more than 32 tiles per CTA (34: 1472 CTAs, whole waves of two
    # CTAs per SM). Its sums must equal, bit for bit, those of 128-candidate
    # launches (3 tiles per CTA), and the oracle's within 1e-6.
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(0)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    rng = np.random.default_rng(3)
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    cands = lo + rng.random((4096, 5)) * (hi - lo)
    full = ctx.objective(cands, pt.TIER_F64)
    for k0 in (0, 1984, 3968):
        part = ctx.objective(cands[k0:k0 + 128].copy(), pt.TIER_F64)
        assert np.array_equal(part, full[k0:k0 + 128])
    idx = np.arange(0, 4096, 256)
    want = oracle.sse_many(blk.values(), blk.fs, blk.t0, cands[idx])
    assert np.max(_rel(full[idx], want)) <= 1e-6


def test_device_pointers_and_torch_stream(ctx):
    import torch
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(9, n=30_000)
    dev = torch.from_numpy(blk.samples).cuda()
    ctx.load_block(dev, blk.fs, blk.t0, blk.scale)
    cands = _candidates(blk, np.random.default_rng(1), nrand=3)
    host = ctx.objective(cands, pt.TIER_F64)
    dc = torch.from_numpy(cands).cuda()
    out = ctx.objective(dc, pt.TIER_F64)
    assert np.array_equal(out.cpu().numpy(), host)


def test_invalid_arguments(ctx):
    import paper_1906_10598_b300 as pt
    with pytest.raises(pt.PhaseTrackError) as e:
        ctx.load_block(np.zeros(10), 0.0, 0.0)
    assert e.value.code == pt.PT_EINVAL
    with pytest.raises(pt.PhaseTrackError) as e:
        ctx.objective(np.zeros((2, 5)), 7)
    assert e.value.code == pt.PT_EINVAL
    c2 = pt.Context(0)
    with pytest.raises(pt.PhaseTrackError) as e:
        c2.objective(np.zeros((2, 5)))
    assert e.value.code == pt.PT_ENOBLOCK
    c2.close()


@pytest.mark.parametrize("f0_frac", [0.2, 0.45])
def test_phase_generator_error_from_clean_tone(ctx, f0_frac):
    # A noiseless FP64 tone evaluated at its own parameters: the oracle's SSE is
    # ~0, the GPU's is sum (A cos phi - A cos phi_hat)^2 ~ A^2 sum sin^2(phi) d^2,
    # so sqrt(2 SSE / (N A^2)) is the RMS error of the phase generator and
    # cosine together, over every sample of the block (paper-size block; f0 at
    # 0.2 fs as in the paper's range, and at 0.45 fs near Nyquist).
    import paper_1906_10598_b300 as pt
    n, fs = 400_000, 10_000.0
    t0 = synth.centred_t0(n, fs)
    truth = np.array([1.0, 0.7, f0_frac * fs, 4.2, 0.04])
    s = synth.clean_tone(truth, n, fs, t0)
    assert oracle.sse(s, fs, t0, truth) < 1e-18 * n
    ctx.load_block(s, fs, t0)
    rms = {}
    for name, tier in (("f64", pt.TIER_F64), ("plain", pt.TIER_PLAIN), ("df32", pt.TIER_DF32), ("f32", pt.TIER_F32)):
        sse = float(ctx.objective(truth[None, :], tier)[0])
        rms[name] = np.sqrt(2.0 * sse / (n * truth[0] ** 2))
    print("phase+cos RMS error (rad):", {k: f"{v:.2e}" for k, v in rms.items()})
    assert rms["plain"] <= 1e-9
    assert rms["f64"] <= 1e-6
    assert rms["df32"] <= 1e-6
