"""Bounded device-side waits (GPU).

* The DE exchange: a launch whose last CTA is not started
  (pt_inject_missing_cta, host side) leaves every other CTA's exchange wait
  without its last arrival.
* The sample staging: with pt_inject_short_tx (host side) each CTA's staging
  mbarrier expects 16 bytes more than its bulk copies bring, so its wait
  cannot complete.

Each wait gives up after the context's limit (pt_set_wait_timeout), the
kernel returns, the call reports PT_ETIMEOUT, and the context stays usable:
the next result is the same as before the failure. No fault, trap or
unbounded wait is involved."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    c = pt.Context(0)
    yield c
    c.inject_missing_cta(False)
    c.inject_short_tx(False)
    c.close()


def test_exchange_wait_runs_out_and_the_context_recovers(ctx):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(0, n=40_000)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ref = ctx.de_solve(blk.bounds, 32, 20, 0.7, 0.9, 3, pt.TIER_F64)
    try:
        ctx.set_wait_timeout(0.05)
        ctx.inject_missing_cta(True)
        t = time.perf_counter()
        with pytest.raises(pt.PhaseTrackError) as e:
            ctx.de_solve(blk.bounds, 32, 20, 0.7, 0.9, 3, pt.TIER_F64)
        assert e.value.code == pt.PT_ETIMEOUT
        assert time.perf_counter() - t < 10.0
    finally:
        ctx.inject_missing_cta(False)
        ctx.set_wait_timeout(2.0)
    again = ctx.de_solve(blk.bounds, 32, 20, 0.7, 0.9, 3, pt.TIER_F64)
    assert np.array_equal(again[0], ref[0]) and again[1] == ref[1]
    # a one-tile block runs on one CTA, which injection leaves alone
    ctx.load_block(blk.samples[:200], blk.fs, blk.t0, blk.scale)
    ctx.inject_missing_cta(True)
    try:
        p, f = ctx.de_solve(blk.bounds, 16, 5, 0.7, 0.9, 1, pt.TIER_F64)
        assert np.isfinite(f)
    finally:
        ctx.inject_missing_cta(False)


def test_wait_timeout_range(ctx):
    import paper_1906_10598_b300 as pt
    for bad in (0.0, 1e-4, 61.0, float("nan")):
        with pytest.raises(pt.PhaseTrackError):
            ctx.set_wait_timeout(bad)
    ctx.set_wait_timeout(2.0)


def test_staging_wait_runs_out_and_the_context_recovers(ctx):
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(1, n=40_000 + 17)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    ref = ctx.de_solve(blk.bounds, 32, 20, 0.7, 0.9, 3, pt.TIER_F64)
    cands = np.vstack([blk.truth, blk.bounds[:, 0], blk.bounds[:, 1]])
    ref_obj = ctx.objective(cands, pt.TIER_F64)
    try:
        ctx.set_wait_timeout(0.05)
        ctx.inject_short_tx(True)
        for call in (lambda: ctx.de_solve(blk.bounds, 32, 20, 0.7, 0.9, 3, pt.TIER_F64),
                     lambda: ctx.objective(cands, pt.TIER_F64)):
            t = time.perf_counter()
            with pytest.raises(pt.PhaseTrackError) as e:
                call()
            assert e.value.code == pt.PT_ETIMEOUT
            assert time.perf_counter() - t < 10.0
    finally:
        ctx.inject_short_tx(False)
        ctx.set_wait_timeout(2.0)
    again = ctx.de_solve(blk.bounds, 32, 20, 0.7, 0.9, 3, pt.TIER_F64)
    assert np.array_equal(again[0], ref[0]) and again[1] == ref[1]
    assert np.array_equal(ctx.objective(cands, pt.TIER_F64), ref_obj)
