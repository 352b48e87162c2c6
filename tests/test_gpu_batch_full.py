"""Full-size parity of the batched DE on the benchmark's 256-block workload.

synth.batch(0, nblocks=256): N log-uniform in 50K-1M int16 samples, fs 1-50
kHz, pop 32-128, G = ceil(80000 / pop), solved in one persistent launch with
the autotuned shape, as `bench.py --mode batch` runs it (pt.Batch, default
tier).
* Every block: the returned SSE equals the oracle's SSE at the returned
  parameters within 1e-6 relative, plus the propagation of a per-sample FP32
  residual error, as in the full-model objective test.
* 8 sampled blocks (every 32nd from block 16): the fit agrees with the FP64
  oracle's own DE fit with the same draws (tests/golden/batch_oracle_fits.json,
  written by tests/golden/make_batch_oracle.py from the oracle alone) within
  1e-3 rad in phi0 and 1e-5 Hz in f0, wherever the oracle reached the truth's
  basin (its SSE at or below the SSE at the truth).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FITS_PATH = os.path.join(os.path.dirname(__file__), "golden", "batch_oracle_fits.json")


@pytest.fixture(scope="module")
def solved():
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    ctx = pt.Context(0)
    blocks = synth.batch(0, nblocks=256)
    batch = pt.Batch(ctx, blocks, pt.TIER_F64)
    batch.run()
    params, sse = batch.results()
    yield blocks, np.asarray(params), np.asarray(sse)
    batch.close()
    ctx.close()


def test_every_block_sse_matches_oracle(solved):
    blocks, params, sse = solved
    assert params.shape == (256, 5) and np.all(np.isfinite(sse))
    for i, b in enumerate(blocks):
        s = b.values()
        want = oracle.sse(s, b.fs, b.t0, params[i])
        dr = 2e-6 * (float(np.max(np.abs(s))) + abs(params[i][0]))
        tol = 1e-6 * want + 2.0 * math.sqrt(b.n * want) * dr + b.n * dr * dr
        assert abs(sse[i] - want) <= tol, (i, sse[i], want)
        # inside the block's ranges
        assert np.all(params[i] >= b.bounds[:, 0]) and np.all(params[i] <= b.bounds[:, 1]), i


def test_sampled_fits_match_oracle_fits(solved):
    blocks, params, sse = solved
    fits = json.load(open(FITS_PATH))
    assert len(fits) == 8
    compared = 0
    for key, ref in sorted(fits.items(), key=lambda kv: int(kv[0])):
        i = int(key)
        b = blocks[i]
        assert (ref["n"], ref["pop"], ref["gens"]) == (b.n, b.pop, b.gens), key
        if ref["sse"] > ref["sse_truth"] * (1 + 1e-6):
            continue  # the oracle's own DE stopped outside the truth's basin
        o = np.asarray(ref["params"])
        assert abs(math.remainder(params[i][1] - o[1], 2 * math.pi)) < 1e-3, (key, params[i], o)
        assert abs(params[i][2] - o[2]) < 1e-5, (key, params[i], o)
        compared += 1
    assert compared >= 4
