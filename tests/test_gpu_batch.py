"""GPU checks of the batched DE launch (many uneven blocks, one persistent
launch under a CUDA graph): every block's fit is bit-identical to the same
block solved alone, for every group size the launch may pick."""
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


def _mixed_blocks():
    blocks = []
    specs = [(3000, synth.I16, 17), (20_000, synth.I8, 40), (70_000, synth.I16, 64), (9_000, synth.F32, 128),
             (41_000, synth.F16, 33), (257, synth.I16, 8), (120_000, synth.I16, 96), (5_000, synth.F64, 24)]
    for i, (n, st, pop) in enumerate(specs):
        b = synth.paper400k(100 + i, n=n, fs=5_000.0 + 1000 * i, storage=st, pop=pop, gens=25)
        b.block_id = i
        b.de_seed = 7 + i
        blocks.append(b)
    return blocks


def test_batch_bit_identical_to_single_solves(ctx):
    import paper_1906_10598_b300 as pt
    blocks = _mixed_blocks()
    alone = []
    for b in blocks:
        ctx.load_block(b.samples, b.fs, b.t0, b.scale)
        alone.append(ctx.de_solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, pt.TIER_F64, block_id=b.block_id))
    for k in (0, 1, 3, 8):
        batch = pt.Batch(ctx, blocks, pt.TIER_F64, group_ctas=k)
        batch.run()
        params, sse = batch.results()
        for i, (p1, s1) in enumerate(alone):
            assert np.array_equal(params[i], p1), (k, i)
            assert sse[i] == s1, (k, i)
        info = batch.info()
        assert info["nblocks"] == len(blocks) and info["group_ctas"] >= 1
        # a second run of the same batch (graph replay) gives the same fits
        batch.run()
        p2, s2 = batch.results()
        assert np.array_equal(p2, params) and np.array_equal(s2, sse)
        batch.close()


def test_batch_degenerate_blocks_bit_identical_to_single_solves(ctx):
    # a one-sample block at the smallest population, a block of exactly one
    # tile, and a small block at the largest population, in one launch
    import paper_1906_10598_b300 as pt
    blocks = []
    for i, (n, pop) in enumerate([(1, 4), (256, 5), (3000, 128)]):
        b = synth.paper400k(200 + i, n=n, fs=2_000.0, pop=pop, gens=12)
        b.block_id = 40 + i
        b.de_seed = 3 + i
        blocks.append(b)
    alone = []
    for b in blocks:
        ctx.load_block(b.samples, b.fs, b.t0, b.scale)
        alone.append(ctx.de_solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, pt.TIER_F64, block_id=b.block_id))
    for k in (0, 2):
        batch = pt.Batch(ctx, blocks, pt.TIER_F64, group_ctas=k)
        batch.run()
        params, sse = batch.results()
        for i, (p1, s1) in enumerate(alone):
            assert np.array_equal(params[i], p1) and sse[i] == s1, (k, i)
        batch.close()


def test_batch_fits_match_oracle_objective(ctx):
    import paper_1906_10598_b300 as pt
    blocks = synth.batch(3, nblocks=6, n_lo=20_000, n_hi=80_000, evals=6_000)
    batch = pt.Batch(ctx, blocks, pt.TIER_F64)
    batch.run()
    params, sse = batch.results()
    info = batch.info()
    assert info["predicted_ms"] > 0 and info["tune_rate"] > 0
    for i, b in enumerate(blocks):
        want = oracle.sse(b.values(), b.fs, b.t0, params[i])
        assert sse[i] == pytest.approx(want, rel=1e-6)
        assert np.all(params[i] >= b.bounds[:, 0] - 1e-12) and np.all(params[i] <= b.bounds[:, 1] + 1e-12)
    batch.close()


def test_batch_invalid(ctx):
    import paper_1906_10598_b300 as pt
    b = synth.paper400k(1, n=1000, gens=3)
    b.pop = 3
    with pytest.raises(pt.PhaseTrackError):
        pt.Batch(ctx, [b])


def test_full_model_batch_bit_identical_to_single_solves(ctx):
    # the full model's blocks (amplitude slope, order-4 phase) in one launch:
    # every fit equals pt_de_solve_full on the block alone, and its SSE the
    # oracle's evaluation of the returned parameters
    import paper_1906_10598_b300 as pt
    blocks = []
    for i, (n, st, pop) in enumerate([(30_000, synth.I16, 32), (4_000, synth.F32, 48), (77_777, synth.I8, 64),
                                      (257, synth.I16, 8)]):
        b = synth.perigee400k(20 + i, n=n, storage=st, pop=pop, gens=30)
        b.block_id, b.de_seed = 50 + i, 3 + i
        blocks.append(b)
    alone = []
    for b in blocks:
        ctx.load_block(b.samples, b.fs, b.t0, b.scale)
        alone.append(ctx.de_solve_full(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, block_id=b.block_id))
    for k in (0, 2):
        batch = pt.Batch(ctx, blocks, group_ctas=k)
        batch.run()
        params, sse = batch.results()
        assert params.shape == (len(blocks), 7)
        for i, (p1, s1) in enumerate(alone):
            assert np.array_equal(params[i], p1) and sse[i] == s1, (k, i)
        batch.close()
    for i, b in enumerate(blocks[:2]):
        assert sse[i] == pytest.approx(oracle.sse_full(b.values(), b.fs, b.t0, params[i]), rel=1e-6)
    # the cubic and full models do not mix in one batch
    with pytest.raises(ValueError):
        pt.Batch(ctx, [blocks[0], synth.paper400k(1, n=1000, gens=3)])


@pytest.mark.parametrize("strategy", ["best1jitter", "eitheror"])
def test_batch_strategies_bit_identical_to_single_solves(ctx, strategy):
    import paper_1906_10598_b300 as pt
    blocks = _mixed_blocks()[:5]
    ctx.set_strategy(strategy)
    try:
        alone = []
        for b in blocks:
            ctx.load_block(b.samples, b.fs, b.t0, b.scale)
            alone.append(ctx.de_solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, pt.TIER_F64,
                                      block_id=b.block_id))
        batch = pt.Batch(ctx, blocks, pt.TIER_F64, group_ctas=4)
        batch.run()
        params, sse = batch.results()
        for i, (p1, s1) in enumerate(alone):
            assert np.array_equal(params[i], p1) and sse[i] == s1, i
        batch.close()
    finally:
        ctx.set_strategy("rand1bin")
