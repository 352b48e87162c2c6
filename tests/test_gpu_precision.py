"""Full-size DE parity against stored oracle fits: N = 400,000 samples at
10 kHz, pop 64, 1250 generations (the benchmark's workload and launch
configuration), stored as int8, FP16 and FP32.

tests/golden/precision_oracle_fits.json holds the FP64 oracle's own fits of
these blocks, written by tests/golden/make_precision_oracle.py, which calls
only the oracle and the input generators (each fit takes the oracle minutes
of host time). The default tier's fit must agree with the oracle's within the
fit tolerances (phi0 within 1e-3 rad, f0 within 1e-5 Hz) wherever the
oracle reached the global basin (its SSE at or below the truth's), and its
SSE must match the oracle's evaluation of the same parameters within 1e-6.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FITS_PATH = os.path.join(os.path.dirname(__file__), "golden", "precision_oracle_fits.json")
FITS = json.load(open(FITS_PATH)) if os.path.exists(FITS_PATH) else {}


@pytest.fixture(scope="module")
def ctx():
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    c = pt.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("storage", ["i8", "f16", "f32"])
def test_full_size_fits_match_stored_oracle_fits(ctx, storage):
    import paper_1906_10598_b300 as pt
    keys = sorted((k for k in FITS if k.startswith(storage + "/")), key=lambda k: int(k.split("/")[1]))
    if not keys:
        pytest.skip("no stored oracle fits")
    compared = 0
    for key in keys:
        ref = FITS[key]
        seed = int(key.split("/")[1])
        blk = synth.precision(seed, synth.STORAGE_NAMES[storage])
        ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
        p, f = ctx.de_solve(blk.bounds, blk.pop, blk.gens, blk.F, blk.CR, blk.de_seed, pt.TIER_F64)
        assert f == pytest.approx(oracle.sse(blk.values(), blk.fs, blk.t0, p), rel=1e-6), key
        if ref["sse"] > ref["sse_truth"] * (1 + 1e-6):
            continue  # the oracle's own DE stopped outside the truth's basin
        o = np.asarray(ref["params"])
        assert abs(math.remainder(p[1] - o[1], 2 * math.pi)) < 1e-3, (key, p, o)
        assert abs(p[2] - o[2]) < 1e-5, (key, p, o)
        compared += 1
    assert compared >= len(keys) // 2
