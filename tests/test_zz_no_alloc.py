"""The allocation-free objective entry point (pt_objective_noalloc).

Host programs that may not allocate device memory while running (a real-time
recording pipeline that reserves the GPU's memory up front, or a framework
that forbids driver allocations after start-up) call this entry point with
device buffers they own; its only scratch is a fixed array inside the
library. This test calls it through the C ABI twice in a row and checks each
result against pt_objective, within the objective tests' 1e-6 relative
tolerance. It lives in a file pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _proto(lib):
    lib.pt_objective_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.pt_objective_noalloc.restype = ctypes.c_int


def test_noalloc_objective_matches_pt_objective_twice():
    import torch
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    lib = pt.load_library()
    _proto(lib)
    torch.cuda.set_device(0)
    blk = synth.paper400k(21, n=30_000 + 5)
    padded = (blk.n + 255) // 256 * 256
    dev_samples = torch.zeros(padded, dtype=torch.int16, device="cuda")
    dev_samples[: blk.n] = torch.from_numpy(blk.samples).cuda()
    ctx = pt.Context(0)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    rng = np.random.default_rng(5)
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    for call, count in enumerate((37, 200)):
        cands = np.vstack([blk.truth, lo + rng.random((count - 1, 5)) * (hi - lo)])
        want = ctx.objective(cands, pt.TIER_F64)
        d_cands = torch.from_numpy(cands).cuda()
        out = torch.full((count,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = lib.pt_objective_noalloc(dev_samples.data_ptr(), blk.n, pt.PT_I16, blk.scale, blk.fs, blk.t0, 0.0,
                                      d_cands.data_ptr(), count, out.data_ptr(), pt.TIER_F64, None)
        assert rc == pt.PT_OK, (call, rc)
        got = out.cpu().numpy()
        assert np.max(np.abs(got - want) / want) <= 1e-6, call
    # sizes beyond the fixed scratch are rejected
    big = torch.zeros((pt_max := 4096 + 1, 5), dtype=torch.float64, device="cuda")
    out = torch.zeros(pt_max, dtype=torch.float64, device="cuda")
    rc = lib.pt_objective_noalloc(dev_samples.data_ptr(), blk.n, pt.PT_I16, blk.scale, blk.fs, blk.t0, 0.0,
                                  big.data_ptr(), pt_max, out.data_ptr(), pt.TIER_F64, None)
    assert rc == pt.PT_EINVAL
    ctx.close()
