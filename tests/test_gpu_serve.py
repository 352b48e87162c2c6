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
