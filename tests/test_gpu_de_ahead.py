"""GPU DE over long runs (Sec. 1.2, Table 3-1-1).

* Against the oracle: a 4096-sample block in the all-FP64 tier, whose
  objective agrees with the oracle's to ~1e-12, keeps its population identical
  to the oracle's synchronous DE (the same draws and FP64 trial arithmetic)
  for hundreds of generations, until a selection compares two values closer
  than that (here between generations 250 and 300 for the chi-square, 150 and
  200 for the correlation objective).
* Building the next generation ahead: on the 400K block (148 CTAs, resident
  tiles, warps that finish the evaluation early) the late generations replace
  at most one individual, so their trials and set-up are built ahead and the
  stale ones rebuilt after the selection. The same fit through a batch of one
  CTA per block, which streams its tiles and never builds ahead, must give the
  same bits.
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
    c.set_strategy("rand1bin")
    c.set_objective("chi2")
    c.close()


@pytest.mark.parametrize("strategy,objective,horizon", [("rand1bin", "chi2", 250), ("eitheror", "chi2", 200),
                                                        ("rand1bin", "cor", 150)])
def test_long_runs_match_the_oracle(ctx, strategy, objective, horizon):
    import paper_1906_10598_b300 as pt
    blk = synth.single4096(11)
    b = blk.bounds.copy()
    if objective == "cor":
        b[0] = (blk.truth[0], blk.truth[0])  # Eq. 2-2-6's model holds the amplitude
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ctx.set_strategy(strategy)
    ctx.set_objective(objective)
    try:
        for gens in (horizon // 2, horizon):
            _, _, gpop, gfit = ctx.de_solve(b, 32, gens, 0.7, 0.9, 21, pt.TIERS["plain"], return_population=True)
            _, _, opop, ofit = oracle.de_solve(blk.values(), blk.fs, blk.t0, b, 32, gens, 0.7, 0.9, 21,
                                               return_population=True, objective=objective, strategy=strategy)
            same = np.all(gpop == opop, axis=1)
            assert same.all(), (strategy, objective, gens, np.where(~same))
            if objective == "cor":
                # the cross-correlations behind F_cor, against their scale n smax A
                cg, co = np.tan(1 / gfit - np.pi / 2), np.tan(1 / ofit - np.pi / 2)
                scale = blk.n * float(np.max(np.abs(blk.values()))) * blk.truth[0]
                assert np.all(np.abs(cg - co) <= 1e-9 * scale)
            else:
                assert np.all(np.abs(gfit - ofit) <= 1e-9 * ofit)
    finally:
        ctx.set_strategy("rand1bin")
        ctx.set_objective("chi2")


@pytest.mark.parametrize("strategy", ["rand1bin", "eitheror"])
def test_built_ahead_bit_identical_to_a_launch_that_never_builds_ahead(ctx, strategy):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(0)
    gens, seed = 400, 5
    ctx.set_strategy(strategy)
    try:
        ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
        p1, s1, pop1, _ = ctx.de_solve(blk.bounds, 64, gens, 0.7, 0.9, seed, pt.TIER_F64, return_population=True)
        # the regime: between the last generations at most one member changed
        _, _, pop0, _ = ctx.de_solve(blk.bounds, 64, gens - 1, 0.7, 0.9, seed, pt.TIER_F64, return_population=True)
        assert (~np.all(pop0 == pop1, axis=1)).sum() <= 1
        blk.pop, blk.gens, blk.F, blk.CR, blk.de_seed, blk.block_id = 64, gens, 0.7, 0.9, seed, 0
        batch = pt.Batch(ctx, [blk], pt.TIER_F64, group_ctas=1)
        try:
            assert batch.info()["group_ctas"] == 1
            batch.run()
            params, sse = batch.results()
        finally:
            batch.close()
        assert np.array_equal(params[0], p1) and sse[0] == s1
    finally:
        ctx.set_strategy("rand1bin")
