"""GPU checks of the serving loop (pt_submit / pt_poll): blocks from several
station streams submitted while others run are admitted as slots free up,
and every fit is bit-identical to the same block solved alone."""
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
    c.close()


def _stream_blocks(nper=3):
    out = []
    for spec in synth.make_streams(11, fs_list=(10_000.0, 20_000.0, 35_000.0, 50_000.0), block_range=(0.3, 1.2)):
        for k in range(nper):
            b = synth.stream_block(spec, k)
            b.gens = 40
            out.append((spec.stream_id, b))
    return out


def _wait(server, tickets, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t not in res:
                r = server.poll(t)
                if r is not None:
                    res[t] = r
        time.sleep(0.001)
    return res


def test_served_fits_bit_identical_to_alone(ctx):
    import paper_1906_10598_b300 as pt
    blocks = _stream_blocks()
    alone = []
    for sid, b in blocks:
        ctx.load_block(b.samples, b.fs, b.t0, b.scale)
        alone.append(ctx.de_solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, pt.TIER_F64, block_id=b.block_id))
    server = pt.Server(ctx, max_inflight=3, ctas_per_request=16, max_queued=64)
    tickets = []
    for i, (sid, b) in enumerate(blocks):
        t = server.submit(b, pt.TIER_F64, stream_id=sid)
        assert t is not None
        tickets.append(t)
        if i % 4 == 3:
            time.sleep(0.002)  # later blocks arrive while earlier ones run
    res = _wait(server, tickets)
    assert len(res) == len(tickets)
    for (sid, b), (p1, s1), t in zip(blocks, alone, tickets):
        r = res[t]
        assert r["status"] == pt.PT_OK and r["stream_id"] == sid
        assert np.array_equal(r["params"], p1) and r["sse"] == s1
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
    # polled results are released; unknown tickets are errors
    with pytest.raises(pt.PhaseTrackError):
        server.poll(tickets[0])


def test_queue_backpressure_and_small_budget(ctx):
    import paper_1906_10598_b300 as pt
    blocks = _stream_blocks(2)
    # one slot, room for a single block's samples, a queue of 2
    budget = max(b.samples.nbytes for _, b in blocks) + 1024
    server = pt.Server(ctx, max_inflight=1, ctas_per_request=8, mem_budget_bytes=budget, max_queued=2)
    tickets, refused = [], 0
    for sid, b in blocks:
        t = server.submit(b, pt.TIER_F64, stream_id=sid)
        if t is None:
            refused += 1
        else:
            tickets.append(t)
    assert refused > 0  # PT_EAGAIN once the queue is full
    res = _wait(server, tickets)
    assert len(res) == len(tickets) and all(r["status"] == pt.PT_OK for r in res.values())


def test_served_full_model_requests_bit_identical_to_alone():
    # cubic and full-model requests (7 x 2 bounds) mixed in one serving loop
    import paper_1906_10598_b300 as pt
    c = pt.Context(0)
    try:
        blocks = []
        for k in range(3):
            blocks.append(synth.perigee400k(30 + k, n=20_000 + 999 * k, gens=40))
            blocks.append(synth.paper400k(40 + k, n=15_000 + 777 * k, gens=40))
        for i, b in enumerate(blocks):
            b.block_id, b.de_seed = 200 + i, 9 + i
        alone = []
        for b in blocks:
            c.load_block(b.samples, b.fs, b.t0, b.scale)
            if b.bounds.shape[0] == 7:
                alone.append(c.de_solve_full(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, block_id=b.block_id))
            else:
                alone.append(c.de_solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, pt.TIER_F64,
                                        block_id=b.block_id))
        server = pt.Server(c, max_inflight=2, ctas_per_request=16, max_queued=16)
        tickets = [server.submit(b, pt.TIER_F64, stream_id=i) for i, b in enumerate(blocks)]
        assert all(t is not None for t in tickets)
        res = _wait(server, tickets)
        assert len(res) == len(tickets)
        for t, (p1, s1), b in zip(tickets, alone, blocks):
            r = res[t]
            assert r["status"] == 0 and len(r["params"]) == b.bounds.shape[0]
            assert np.array_equal(r["params"], p1) and r["sse"] == s1
    finally:
        c.close()


def test_serving_loop_takes_the_context_objective():
    # the loop starts with the context's objective (the correlation objective
    # here): served fits equal the context's own solves on it, and full-model
    # requests, which run on the chi-square only, are refused
    import paper_1906_10598_b300 as pt
    c = pt.Context(0)
    try:
        c.set_objective("cor")
        blk = synth.paper400k(3, n=20_000, gens=30)
        b = blk.bounds.copy()
        b[0] = (blk.truth[0], blk.truth[0])
        c.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
        p1, s1 = c.de_solve(b, blk.pop, blk.gens, blk.F, blk.CR, blk.de_seed, pt.TIER_F64, block_id=blk.block_id)
        server = pt.Server(c, max_inflight=1, ctas_per_request=16)
        t = server.submit(blk, pt.TIER_F64, bounds=b)
        r = _wait(server, [t])[t]
        assert r["status"] == 0 and np.array_equal(r["params"], p1) and r["sse"] == s1
        with pytest.raises(pt.PhaseTrackError):
            server.submit(synth.perigee400k(1, n=5_000, gens=5))
    finally:
        c.set_objective("chi2")
        c.close()
