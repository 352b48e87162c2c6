"""The allocation-free objective entry point (pt_objective_noalloc).

Host programs that may not allocate device memory while running (a real-time
recording pipeline that reserves the GPU's memory up front, or a framework
that forbids driver allocations after start-up) call this entry point with
device buffers they own; its only scratch is a fixed array inside the
library. These tests call it through the C ABI twice in a row for every
precision tier and sample type, and check each result against pt_objective
(1e-6 relative, the objective tests' tolerance) and against the FP64 oracle
(the tier's own tolerance). Buffers the kernels could not use (misaligned,
too short for the whole tiles the staging reads, host memory, a float type
without a bound) are refused on the host before anything is launched. The
file is collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# tolerance of each tier against the oracle (as in the objective tests); the
# naive FP32 tier is reported, not bounded
ORACLE_TOL = {0: 1e-6, 1: 1e-9, 2: 1e-5}


def _proto(lib):
    lib.pt_objective_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.pt_objective_noalloc.restype = ctypes.c_int


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    lib = pt.load_library()
    _proto(lib)
    torch.cuda.set_device(0)
    ctx = pt.Context(0)
    yield pt, lib, ctx
    ctx.close()


def _device_samples(blk):
    """The block's stored samples on the device, zero-padded to whole 256-sample tiles."""
    import torch
    padded = (blk.n + 255) // 256 * 256
    tdt = {np.dtype(np.int8): torch.int8, np.dtype(np.int16): torch.int16, np.dtype(np.float16): torch.float16,
           np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}[blk.samples.dtype]
    dev = torch.zeros(padded, dtype=tdt, device="cuda")
    dev[: blk.n] = torch.from_numpy(blk.samples).cuda()
    return dev


def _call(lib, pt, dev_samples, blk, smax, d_cands, count, out, tier):
    return lib.pt_objective_noalloc(dev_samples.data_ptr(), blk.n, blk.dtype, blk.scale, blk.fs, blk.t0, smax,
                                    d_cands.data_ptr(), count, out.data_ptr(), tier, None)


@pytest.mark.parametrize("storage", ["i16", "i8", "f16", "f32", "f64"])
@pytest.mark.parametrize("tier", [0, 1, 2, 3])
def test_noalloc_matches_pt_objective_and_oracle_twice(env, storage, tier):
    import torch
    pt, lib, ctx = env
    blk = synth.paper400k(21, n=30_000 + 5, storage=synth.STORAGE_NAMES[storage])
    dev_samples = _device_samples(blk)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    vals = blk.values()
    # float samples need a stated bound (FP16's type range, 65504 x scale, is
    # far above these samples and would coarsen the fixed-point sums); the
    # integer types, quantised to their full range, take the type's range (0)
    smax = float(np.max(np.abs(vals))) if storage in ("f16", "f32", "f64") else 0.0
    rng = np.random.default_rng(5 + tier)
    lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
    for call, count in enumerate((37, 200)):
        cands = np.vstack([blk.truth, lo + rng.random((count - 1, 5)) * (hi - lo)])
        want_ctx = ctx.objective(cands, tier)
        d_cands = torch.from_numpy(cands).cuda()
        out = torch.full((count,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = _call(lib, pt, dev_samples, blk, smax, d_cands, count, out, tier)
        assert rc == pt.PT_OK, (call, rc)
        got = out.cpu().numpy()
        assert np.max(np.abs(got - want_ctx) / want_ctx) <= 1e-6, (call, tier)
        if tier in ORACLE_TOL:
            idx = np.arange(0, count, 9)
            want = oracle.sse_many(vals, blk.fs, blk.t0, cands[idx])
            assert np.max(np.abs(got[idx] - want) / want) <= ORACLE_TOL[tier], (call, tier)
        else:
            assert np.all(np.isfinite(got))


def _allocation_end(ptr):
    """End address of the device allocation holding ``ptr`` (driver query)."""
    cu = ctypes.CDLL("libcuda.so.1")
    cu.cuMemGetAddressRange_v2.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_size_t),
                                           ctypes.c_uint64]
    cu.cuMemGetAddressRange_v2.restype = ctypes.c_int
    base, size = ctypes.c_uint64(0), ctypes.c_size_t(0)
    assert cu.cuMemGetAddressRange_v2(ctypes.byref(base), ctypes.byref(size), ctypes.c_uint64(ptr)) == 0
    return base.value + size.value


def test_noalloc_rejects_unusable_buffers_on_the_host(env):
    import torch
    pt, lib, ctx = env
    blk = synth.paper400k(3, n=1000)  # int16, 4 tiles (1024 samples staged)
    dev_samples = _device_samples(blk)
    cands = torch.from_numpy(np.vstack([blk.truth] * 4)).cuda()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert _call(lib, pt, dev_samples, blk, 0.0, cands, 4, out, 0) == pt.PT_OK
    first = out.clone()

    def rc_of(samples_ptr, n=blk.n, dtype=blk.dtype, smax=0.0, cand_ptr=None, count=4, out_ptr=None):
        return lib.pt_objective_noalloc(samples_ptr, n, dtype, blk.scale, blk.fs, blk.t0, smax,
                                        cand_ptr if cand_ptr is not None else cands.data_ptr(), count,
                                        out_ptr if out_ptr is not None else out.data_ptr(), 0, None)

    # a sample pointer off the 16-byte alignment the bulk copies need
    assert rc_of(dev_samples.data_ptr() + 2) == pt.PT_EINVAL
    # samples that end 1024 bytes before their allocation does: 512 int16
    # samples (two whole tiles) fit, 600 (three tiles staged) would be read past the end
    tail = (_allocation_end(dev_samples.data_ptr()) - 1024) & ~15
    assert _allocation_end(dev_samples.data_ptr()) - tail < 1536
    assert rc_of(tail, n=600) == pt.PT_EINVAL
    assert rc_of(tail, n=500) == pt.PT_OK
    # candidate rows and outputs past their allocations' ends
    c_end = _allocation_end(cands.data_ptr())
    assert rc_of(dev_samples.data_ptr(), cand_ptr=c_end - 40, count=1, out_ptr=out.data_ptr()) == pt.PT_OK
    assert rc_of(dev_samples.data_ptr(), cand_ptr=c_end - 40, count=4) == pt.PT_EINVAL
    o_end = _allocation_end(out.data_ptr())
    assert rc_of(dev_samples.data_ptr(), count=4, out_ptr=o_end - 8) == pt.PT_EINVAL
    # host memory for the samples, the candidates or the output
    host = np.zeros(1024, dtype=np.int16)
    assert rc_of(host.ctypes.data) == pt.PT_EINVAL
    hc = np.vstack([blk.truth] * 4)
    assert rc_of(dev_samples.data_ptr(), cand_ptr=hc.ctypes.data) == pt.PT_EINVAL
    ho = np.zeros(4)
    assert rc_of(dev_samples.data_ptr(), out_ptr=ho.ctypes.data) == pt.PT_EINVAL
    # a float sample type with no stated bound
    f32 = torch.zeros(1024, dtype=torch.float32, device="cuda")
    assert rc_of(f32.data_ptr(), dtype=pt.PT_F32, smax=0.0) == pt.PT_EINVAL
    # a candidate count beyond the fixed scratch
    big = torch.zeros((4097, 5), dtype=torch.float64, device="cuda")
    bout = torch.zeros(4097, dtype=torch.float64, device="cuda")
    assert rc_of(dev_samples.data_ptr(), cand_ptr=big.data_ptr(), count=4097, out_ptr=bout.data_ptr()) == \
        pt.PT_EINVAL
    # nothing above was launched with a bad buffer: the entry point still gives the same result
    assert _call(lib, pt, dev_samples, blk, 0.0, cands, 4, out, 0) == pt.PT_OK
    assert torch.equal(out, first)
