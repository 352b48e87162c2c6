"""Replica routing for N > 1 GPUs, tested with CPU processes standing in for ranks.

Blocks are independent, so N GPUs run N replicas with no collective on the
data path: the router assigns each block to one rank, each rank fits its own
blocks, and rank 0 gathers the results and the slowest rank's time. Here the
ranks are world-size-2 gloo processes on the CPU and the per-block solver is
the CPU oracle (the GPU path runs the same host logic around pt_de_solve).
"""
import json
import os
import socket

import numpy as np
import pytest

from paper_1906_10598_b300 import replicas


def test_assign_covers_every_unit_once():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        costs = rng.integers(1, 100, size=37).astype(float)
        parts = replicas.assign(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        for p in parts:
            assert p == sorted(p)


def test_assign_balances_by_cost():
    # LPT: the heaviest rank carries at most the mean load plus one unit
    rng = np.random.default_rng(4)
    costs = rng.uniform(1.0, 10.0, size=200)
    parts = replicas.assign(costs, 4)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= np.mean(loads) + costs.max() + 1e-9


def test_assign_equal_costs_round_robin_and_deterministic():
    assert replicas.assign([1.0] * 4, 4) == [[0], [1], [2], [3]]
    assert replicas.assign([5.0, 1.0, 1.0], 2) == [[0], [1, 2]]
    c = [3.0, 3.0, 2.0, 2.0, 1.0]
    assert replicas.assign(c, 2) == replicas.assign(list(c), 2)
    with pytest.raises(ValueError):
        replicas.assign([1.0], 0)
    with pytest.raises(ValueError):
        replicas.assign([float("nan")], 1)
    with pytest.raises(ValueError):
        replicas.my_units([1.0], 2, 2)


def _tiny_blocks():
    import synth
    blocks = []
    for seed in range(5):
        b = synth.paper400k(seed, n=64 * (seed + 1), fs=200.0, gens=6)
        blocks.append(b)
    return blocks


def _solve(b):
    import oracle
    p, f = oracle.de_solve(b.values(), b.fs, b.t0, b.bounds, 8, b.gens, b.F, b.CR, b.de_seed, nthreads=1)
    return [float(v) for v in p], float(f)


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        blocks = _tiny_blocks()
        costs = [b.n * 8 * (b.gens + 1) for b in blocks]
        mine = replicas.my_units(costs, world, rank)
        results = {i: _solve(blocks[i]) for i in mine}
        gathered = replicas.gather(results)
        slowest = replicas.max_over_ranks(float(rank + 1))
        if rank == 0:
            merged = {}
            for part in gathered:
                for i, r in part.items():
                    assert i not in merged
                    merged[i] = r
            with open(out_path, "w") as fh:
                json.dump({"merged": {str(k): v for k, v in merged.items()}, "slowest": slowest,
                           "parts": [sorted(p) for p in gathered]}, fh)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_replicas_match_single_process(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "replicas.json")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = json.load(open(out))
    blocks = _tiny_blocks()
    # every block solved exactly once, by the rank the router chose
    costs = [b.n * 8 * (b.gens + 1) for b in blocks]
    want_parts = replicas.assign(costs, 2)
    assert [sorted(map(int, p)) for p in got["parts"]] == want_parts
    assert sorted(map(int, got["merged"])) == list(range(len(blocks)))
    # same fits as one process solving every block
    for i, b in enumerate(blocks):
        p, f = _solve(b)
        gp, gf = got["merged"][str(i)]
        assert np.array_equal(np.array(gp), np.array(p)) and gf == f
    # the job time is the slowest rank's
    assert got["slowest"] == 2.0
