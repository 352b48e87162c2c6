"""GPU parity of the correlation objective (Eq. 2-2-5 with the constant-amplitude
model of Eq. 2-2-6) against the FP64 oracle.

* pt_objective on PT_OBJ_COR: F_cor within 1e-6 relative of the oracle for
  random, true and far candidates, and the cross-correlation behind it,
  recovered as tan(1/F - pi/2), within 2e-6 of the oracle's relative to
  n * smax * A (F_cor is flat near 1/pi, where only cor shows the error);
* the per-candidate value is independent of the batch it is evaluated in
  (signed fixed-point sums);
* DE on PT_OBJ_COR with A held constant reaches the oracle's fit within
  1e-3 rad in phi0 and 1e-5 Hz in f0; the initial population is bit-identical;
* the comparison tiers: the all-FP64 tier's cross-correlation within 1e-9 and
  the double-float tier's within 2e-6 of n smax A, the all-FP64 tier's DE
  populations bit-identical to the oracle's in the early generations.
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
    c.set_objective("chi2")
    c.close()


def _cands(blk, rng, A):
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    rows = [lo + rng.random(5) * (hi - lo) for _ in range(20)]
    rows.append(np.array(blk.truth, dtype=np.float64))
    far = np.array(blk.truth, dtype=np.float64)
    far[2] += 37.0
    rows.append(far)
    c = np.array(rows)
    c[:, 0] = A
    return c


@pytest.mark.parametrize("n", [4096, 50_000, 333_333])
def test_cor_objective_matches_oracle(ctx, n):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(11, n=n)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ctx.set_objective("cor")
    try:
        A = float(blk.truth[0])
        c = _cands(blk, np.random.default_rng(n), A)
        got = ctx.objective(c, pt.TIER_F64)
        want = oracle.cor_objective_many(blk.values(), blk.fs, blk.t0, c)
        # F_cor is as sensitive as cor itself where cor is large and negative
        # (F ~ |cor|) and flat where it is large and positive (F ~ 1/pi): the
        # objective's relative tolerance is the chi-square's, 1e-6
        assert np.max(np.abs(got - want) / want) <= 1e-6, np.max(np.abs(got - want) / want)
        # the cross-correlation behind each value
        cor_g = np.tan(1.0 / got - math.pi / 2)
        cor_o = np.array([oracle.cor(blk.values(), blk.fs, blk.t0, r) for r in c])
        bound = n * float(np.max(np.abs(blk.values()))) * A
        sel = np.abs(cor_o) < 1e6  # outside saturation tan() is well conditioned
        assert np.all(np.abs(cor_g[sel] - cor_o[sel]) <= 2e-6 * bound)
        # chi-square is untouched by the setting once it is switched back
        ctx.set_objective("chi2")
        sse = ctx.objective(c, pt.TIER_F64)
        assert np.max(np.abs(sse - oracle.sse_many(blk.values(), blk.fs, blk.t0, c)) / sse) <= 2e-6
    finally:
        ctx.set_objective("chi2")


def test_cor_objective_independent_of_batch_shape(ctx):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(6, n=50_000)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ctx.set_objective("cor")
    try:
        c = _cands(blk, np.random.default_rng(1), float(blk.truth[0]))
        c = np.concatenate([c] * 10)
        full = ctx.objective(c, pt.TIER_F64)
        for k in (1, 5, 37):
            assert np.array_equal(ctx.objective(c[:k].copy(), pt.TIER_F64), full[:k])
    finally:
        ctx.set_objective("chi2")


@pytest.mark.parametrize("tier,tol", [("plain", 1e-9), ("df32", 2e-6), ("f32", None)])
def test_cor_comparison_tiers(ctx, tier, tol):
    # the all-FP64 and double-float tiers against the oracle (cross-correlation
    # relative to n smax A); the naive FP32 tier is reported, not bounded
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(11, n=50_000)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ctx.set_objective("cor")
    try:
        A = float(blk.truth[0])
        c = _cands(blk, np.random.default_rng(5), A)
        got = ctx.objective(c, pt.TIERS[tier])
        assert np.all(np.isfinite(got)) and np.all(got > 0)
        if tol is None:
            return
        cor_g = np.tan(1.0 / got - math.pi / 2)
        cor_o = np.array([oracle.cor(blk.values(), blk.fs, blk.t0, r) for r in c])
        bound = blk.n * float(np.max(np.abs(blk.values()))) * A
        sel = np.abs(cor_o) < 1e6
        assert np.all(np.abs(cor_g[sel] - cor_o[sel]) <= tol * bound), np.max(np.abs(cor_g[sel] - cor_o[sel])) / bound
    finally:
        ctx.set_objective("chi2")
    with pytest.raises(pt.PhaseTrackError):
        ctx.set_objective(7)


def test_cor_plain_tier_de_bit_identical(ctx):
    import paper_1906_10598_b300 as pt
    blk = synth.single4096(3)
    b = blk.bounds.copy()
    b[0] = (blk.truth[0], blk.truth[0])
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ctx.set_objective("cor")
    try:
        for gens in (0, 1, 6):
            _, _, gpop, gfit = ctx.de_solve(b, 32, gens, 0.7, 0.9, 17, pt.TIER_PLAIN, return_population=True)
            _, _, opop, ofit = oracle.de_solve(blk.values(), blk.fs, blk.t0, b, 32, gens, 0.7, 0.9, 17,
                                               return_population=True, objective="cor")
            same = np.all(gpop == opop, axis=1)
            assert same.sum() >= 31, (gens, np.where(~same))
    finally:
        ctx.set_objective("chi2")


def test_cor_de_fit_matches_oracle(ctx):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(3, n=20_000, gens=300)
    b = blk.bounds.copy()
    b[0] = (blk.truth[0], blk.truth[0])  # the constant "average amplitude" of Eq. 2-2-6
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ctx.set_objective("cor")
    try:
        g, gf = ctx.de_solve(b, 32, 300, 0.7, 0.9, 9, pt.TIER_F64)
        o, of = oracle.de_solve(blk.values(), blk.fs, blk.t0, b, 32, 300, 0.7, 0.9, 9, objective="cor")
        assert g[0] == blk.truth[0]
        assert abs(math.remainder(g[1] - o[1], 2 * math.pi)) < 1e-3 and abs(g[2] - o[2]) < 1e-5
        assert gf == pytest.approx(oracle.cor_objective(blk.values(), blk.fs, blk.t0, g), rel=1e-9)
        # the same DE draws: generation 0 is bit-identical
        _, _, gp, _ = ctx.de_solve(b, 32, 0, 0.7, 0.9, 9, pt.TIER_F64, return_population=True)
        _, _, op, _ = oracle.de_solve(blk.values(), blk.fs, blk.t0, b, 32, 0, 0.7, 0.9, 9, objective="cor",
                                      return_population=True)
        assert np.array_equal(gp, op)
    finally:
        ctx.set_objective("chi2")
