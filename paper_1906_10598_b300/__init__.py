"""Python binding of ``libphasetrack`` (the C ABI in ``include/phasetrack.h``).

Argument marshalling only: every step of the objective and the DE fit runs in
the library's CUDA kernels. Inputs may be numpy arrays (host memory) or torch
CUDA tensors (device memory, passed by pointer); PyTorch is used only as a
carrier of device memory and streams.

The library must be built (``python -m paper_1906_10598_b300.build``); there is
no CPU fallback: if the library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphasetrack.so")

PT_OK, PT_PENDING = 0, 1
PT_EINVAL, PT_ENOMEM, PT_EAGAIN, PT_ETIMEOUT, PT_ECUDA, PT_ENOTCONV, PT_ENOBLOCK = -1, -2, -3, -4, -5, -6, -7
PT_I8, PT_I16, PT_F16, PT_F32, PT_F64 = 0, 1, 2, 3, 4
TIER_F64, TIER_PLAIN, TIER_DF32, TIER_F32 = 0, 1, 2, 3
TIERS = {"f64": TIER_F64, "plain": TIER_PLAIN, "df32": TIER_DF32, "f32": TIER_F32}
OBJ_CHI2, OBJ_COR = 0, 1
OBJECTIVES = {"chi2": OBJ_CHI2, "cor": OBJ_COR}
DE_RAND1_BIN, DE_BEST1_JITTER, DE_EITHER_OR = 0, 3, 6
STRATEGIES = {"rand1bin": DE_RAND1_BIN, "best1jitter": DE_BEST1_JITTER, "eitheror": DE_EITHER_OR}
POP_MAX = 128

_NP_TO_PT = {np.dtype(np.int8): PT_I8, np.dtype(np.int16): PT_I16, np.dtype(np.float16): PT_F16,
             np.dtype(np.float32): PT_F32, np.dtype(np.float64): PT_F64}
_STATUS = {PT_EINVAL: "EINVAL", PT_ENOMEM: "ENOMEM", PT_EAGAIN: "EAGAIN", PT_ETIMEOUT: "ETIMEOUT",
           PT_ECUDA: "ECUDA", PT_ENOTCONV: "ENOTCONV", PT_ENOBLOCK: "ENOBLOCK"}

_lib = None


class PhaseTrackError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class SeedResult(ctypes.Structure):
    """Mirror of ``pt_seed_result``."""
    _fields_ = [("f0", ctypes.c_double), ("f1", ctypes.c_double), ("A", ctypes.c_double), ("piece_len", ctypes.c_int),
                ("peak_bin", ctypes.c_int * 3), ("peak_delta", ctypes.c_double * 3),
                ("piece_freq", ctypes.c_double * 3), ("piece_time", ctypes.c_double * 3),
                ("bounds", ctypes.c_double * 14)]


def load_library():
    """Load libphasetrack.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1906_10598_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, i64, c_int = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int
    lib.pt_create.argtypes = [ctypes.POINTER(vp), c_int]
    lib.pt_create.restype = c_int
    lib.pt_destroy.argtypes = [vp]
    lib.pt_destroy.restype = None
    lib.pt_last_error.argtypes = [vp]
    lib.pt_last_error.restype = ctypes.c_char_p
    lib.pt_set_stream.argtypes = [vp, vp]
    lib.pt_set_stream.restype = c_int
    lib.pt_set_objective.argtypes = [vp, c_int]
    lib.pt_set_objective.restype = c_int
    lib.pt_set_strategy.argtypes = [vp, c_int]
    lib.pt_set_strategy.restype = c_int
    lib.pt_get_stream.argtypes = [vp]
    lib.pt_get_stream.restype = vp
    lib.pt_load_block.argtypes = [vp, vp, i64, c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.pt_load_block.restype = c_int
    lib.pt_objective.argtypes = [vp, vp, i64, vp, c_int]
    lib.pt_objective.restype = c_int
    lib.pt_de_solve.argtypes = [vp, dp, c_int, c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, vp, c_int]
    lib.pt_de_solve.restype = c_int
    lib.pt_de_solve_ex.argtypes = [vp, dp, c_int, c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_uint32, vp, vp, vp, c_int]
    lib.pt_de_solve_ex.restype = c_int
    lib.pt_objective_full.argtypes = [vp, vp, i64, vp, c_int]
    lib.pt_objective_full.restype = c_int
    lib.pt_de_solve_full.argtypes = [vp, dp, c_int, c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint32, vp, vp, vp, c_int]
    lib.pt_de_solve_full.restype = c_int
    lib.pt_last_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.pt_last_kernel_ms.restype = c_int
    lib.pt_seed_bounds.argtypes = [vp, ctypes.c_double, c_int, ctypes.POINTER(SeedResult)]
    lib.pt_seed_bounds.restype = c_int
    lib.pt_set_wait_timeout.argtypes = [vp, ctypes.c_double]
    lib.pt_set_wait_timeout.restype = c_int
    lib.pt_inject_missing_cta.argtypes = [vp, c_int]
    lib.pt_inject_missing_cta.restype = c_int
    lib.pt_inject_short_tx.argtypes = [vp, c_int]
    lib.pt_inject_short_tx.restype = c_int
    _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array or torch tensor (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _is_torch(a) -> bool:
    return hasattr(a, "data_ptr") and not isinstance(a, np.ndarray)


class Context:
    """One ``pt_ctx``: a GPU, its stream, the loaded block and device scratch."""

    def __init__(self, device: int = 0):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        rc = self._lib.pt_create(ctypes.byref(self._h), int(device))
        if rc != PT_OK:
            raise PhaseTrackError(rc, f"pt_create(device={device}) failed")
        self.n = 0

    def close(self):
        if self._h:
            self._lib.pt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def _check(self, rc: int):
        if rc != PT_OK:
            raise PhaseTrackError(rc, (self._lib.pt_last_error(self._h) or b"").decode())

    @property
    def stream(self) -> int:
        return int(self._lib.pt_get_stream(self._h) or 0)

    def set_stream(self, stream_handle: Optional[int]):
        self._check(self._lib.pt_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)))

    def set_strategy(self, strategy):
        """pt_set_strategy: "rand1bin" (default), "best1jitter" ("3") or "eitheror" ("6"), or DE_*."""
        self._check(self._lib.pt_set_strategy(self._h, int(STRATEGIES.get(strategy, strategy))))

    def set_objective(self, objective):
        """pt_set_objective: "chi2" (Eq. 2-2-4) or "cor" (Eq. 2-2-5), or OBJ_*."""
        self._check(self._lib.pt_set_objective(self._h, int(OBJECTIVES.get(objective, objective))))

    def load_block(self, samples, fs: float, t0: float, scale: float = 1.0, dtype: Optional[int] = None):
        """pt_load_block: samples as numpy (host) or torch CUDA tensor (device)."""
        if dtype is None:
            if isinstance(samples, np.ndarray):
                dtype = _NP_TO_PT[samples.dtype]
            else:
                import torch
                dtype = {torch.int8: PT_I8, torch.int16: PT_I16, torch.float16: PT_F16, torch.float32: PT_F32,
                         torch.float64: PT_F64}[samples.dtype]
        n = int(samples.numel() if _is_torch(samples) else samples.size)
        self._check(self._lib.pt_load_block(self._h, ctypes.c_void_p(_ptr(samples)), n, int(dtype), float(scale),
                                            float(fs), float(t0)))
        self.n = n

    @staticmethod
    def _cands_out(cands, dim: int, out):
        if isinstance(cands, np.ndarray):
            c = np.ascontiguousarray(cands, dtype=np.float64).reshape(-1, dim)
            if out is None:
                out = np.zeros(c.shape[0], dtype=np.float64)
        else:
            c = cands.contiguous().reshape(-1, dim)
            if out is None:
                import torch
                out = torch.empty(c.shape[0], dtype=torch.float64, device=c.device)
        return c, c.shape[0], out

    def objective(self, cands, tier: int = TIER_F64, out=None):
        """pt_objective: SSE of each row of ``cands`` (n x 5). Returns ``out``
        (numpy float64 if cands is numpy, else a torch tensor on the same device)."""
        c, n, out = self._cands_out(cands, 5, out)
        self._check(self._lib.pt_objective(self._h, ctypes.c_void_p(_ptr(c)), n, ctypes.c_void_p(_ptr(out)),
                                           int(tier)))
        return out

    def objective_full(self, cands, tier: int = TIER_F64, out=None):
        """pt_objective_full: SSE of each full-model row (A, phi0, f0, f1, f2, A1, f3)."""
        c, n, out = self._cands_out(cands, 7, out)
        self._check(self._lib.pt_objective_full(self._h, ctypes.c_void_p(_ptr(c)), n, ctypes.c_void_p(_ptr(out)),
                                                int(tier)))
        return out

    def de_solve(self, bounds, pop: int, gens: int, F: float, CR: float, seed: int, tier: int = TIER_F64,
                 block_id: int = 0, return_population: bool = False):
        """pt_de_solve_ex: returns (params[5], sse) or (params, sse, population, fitness)."""
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64).reshape(5, 2))
        out = np.zeros(6, dtype=np.float64)
        popv = np.zeros((pop, 5), dtype=np.float64) if return_population else None
        fit = np.zeros(pop, dtype=np.float64) if return_population else None
        self._check(self._lib.pt_de_solve_ex(
            self._h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(pop), int(gens), float(F), float(CR),
            ctypes.c_uint64(int(seed)), ctypes.c_uint32(int(block_id)), ctypes.c_void_p(out.ctypes.data),
            ctypes.c_void_p(popv.ctypes.data if popv is not None else 0),
            ctypes.c_void_p(fit.ctypes.data if fit is not None else 0), int(tier)))
        if return_population:
            return out[:5].copy(), float(out[5]), popv, fit
        return out[:5].copy(), float(out[5])

    def de_solve_full(self, bounds, pop: int, gens: int, F: float, CR: float, seed: int, block_id: int = 0,
                      return_population: bool = False, tier: int = TIER_F64):
        """pt_de_solve_full: the full model's fit; returns (params[7], sse) or
        (params, sse, population[pop, 7], fitness)."""
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64).reshape(7, 2))
        out = np.zeros(8, dtype=np.float64)
        popv = np.zeros((pop, 7), dtype=np.float64) if return_population else None
        fit = np.zeros(pop, dtype=np.float64) if return_population else None
        self._check(self._lib.pt_de_solve_full(
            self._h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(pop), int(gens), float(F), float(CR),
            ctypes.c_uint64(int(seed)), ctypes.c_uint32(int(block_id)), ctypes.c_void_p(out.ctypes.data),
            ctypes.c_void_p(popv.ctypes.data if popv is not None else 0),
            ctypes.c_void_p(fit.ctypes.data if fit is not None else 0), int(tier)))
        if return_population:
            return out[:7].copy(), float(out[7]), popv, fit
        return out[:7].copy(), float(out[7])

    def set_wait_timeout(self, seconds: float):
        """pt_set_wait_timeout: the limit of every bounded device-side wait."""
        self._check(self._lib.pt_set_wait_timeout(self._h, float(seconds)))

    def inject_missing_cta(self, enable: bool):
        """pt_inject_missing_cta: DE launches start one CTA fewer than their
        group (tests of the bounded waits; calls then fail with PT_ETIMEOUT)."""
        self._check(self._lib.pt_inject_missing_cta(self._h, int(bool(enable))))

    def inject_short_tx(self, enable: bool):
        """pt_inject_short_tx: each CTA's sample-staging wait expects 16 bytes
        more than its copies bring (test of that wait's limit; calls then fail
        with PT_ETIMEOUT)."""
        self._check(self._lib.pt_inject_short_tx(self._h, int(bool(enable))))

    def seed_bounds(self, f0_rel: float = 0.1, piece_len: int = 0) -> dict:
        """pt_seed_bounds: the FFT seed of the loaded block's ranges (Sec. 3.1.1);
        ``bounds`` is 7 x 2 (its first 5 rows are the cubic model's)."""
        r = SeedResult()
        self._check(self._lib.pt_seed_bounds(self._h, float(f0_rel), int(piece_len), ctypes.byref(r)))
        return {"f0": r.f0, "f1": r.f1, "A": r.A, "piece_len": r.piece_len, "peak_bin": list(r.peak_bin),
                "peak_delta": list(r.peak_delta), "piece_freq": list(r.piece_freq),
                "piece_time": list(r.piece_time), "bounds": np.array(list(r.bounds)).reshape(7, 2)}

    def last_kernel_ms(self) -> float:
        v = ctypes.c_float()
        self._check(self._lib.pt_last_kernel_ms(self._h, ctypes.byref(v)))
        return float(v.value)


# ---- batched fits ------------------------------------------------------------


class BlockSpec(ctypes.Structure):
    """Mirror of ``pt_block_spec``."""
    _fields_ = [("samples", ctypes.c_void_p), ("n", ctypes.c_int64), ("dtype", ctypes.c_int),
                ("scale", ctypes.c_double), ("fs", ctypes.c_double), ("t0", ctypes.c_double),
                ("bounds", ctypes.c_double * 10), ("pop", ctypes.c_int), ("gens", ctypes.c_int),
                ("F", ctypes.c_double), ("CR", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("block_id", ctypes.c_uint32)]


class Fit(ctypes.Structure):
    """Mirror of ``pt_fit``."""
    _fields_ = [("params", ctypes.c_double * 5), ("sse", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    """Mirror of ``pt_batch_info``."""
    _fields_ = [("nblocks", ctypes.c_int), ("ngroups", ctypes.c_int), ("group_ctas", ctypes.c_int),
                ("tier", ctypes.c_int), ("uses_graph", ctypes.c_int), ("sample_evals", ctypes.c_double),
                ("predicted_ms", ctypes.c_double), ("last_ms", ctypes.c_double), ("tune_rate", ctypes.c_double),
                ("tune_gen_us", ctypes.c_double), ("tune_rate_stream", ctypes.c_double)]


def _batch_protos(lib):
    if getattr(lib, "_batch_protos", False):
        return
    vp = ctypes.c_void_p
    lib.pt_batch_create.argtypes = [vp, ctypes.POINTER(BlockSpec), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(vp)]
    lib.pt_batch_create.restype = ctypes.c_int
    lib.pt_batch_run.argtypes = [vp]
    lib.pt_batch_run.restype = ctypes.c_int
    lib.pt_batch_results.argtypes = [vp, ctypes.POINTER(Fit)]
    lib.pt_batch_results.restype = ctypes.c_int
    lib.pt_batch_create_full.argtypes = [vp, ctypes.POINTER(BlockSpec), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    lib.pt_batch_create_full.restype = ctypes.c_int
    lib.pt_batch_results_full.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.pt_batch_results_full.restype = ctypes.c_int
    lib.pt_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    lib.pt_batch_get_info.restype = ctypes.c_int
    lib.pt_batch_destroy.argtypes = [vp]
    lib.pt_batch_destroy.restype = None
    lib._batch_protos = True


class Batch:
    """``pt_batch``: many blocks solved by one persistent launch.

    ``blocks`` is a sequence of objects with ``samples`` (numpy), ``scale``,
    ``fs``, ``t0``, ``bounds`` (5 x 2, or 7 x 2 for the full model), ``pop``,
    ``gens``, ``F``, ``CR``, ``de_seed`` and ``block_id`` attributes (e.g.
    ``synth.Block``). Blocks with 7 x 2 bounds make a full-model batch
    (``pt_batch_create_full``; all blocks alike)."""

    def __init__(self, ctx: Context, blocks, tier: int = TIER_F64, group_ctas: int = 0):
        self._ctx = ctx
        self._lib = ctx._lib
        _batch_protos(self._lib)
        n = len(blocks)
        specs = (BlockSpec * n)()
        keep = []
        dims = {np.asarray(b.bounds).size // 2 for b in blocks}
        if len(dims) != 1 or dims.pop() not in (5, 7):
            raise ValueError("Batch: every block's bounds must be 5 x 2, or every block's 7 x 2")
        self._dim = np.asarray(blocks[0].bounds).size // 2
        ext = np.zeros((n, 4), dtype=np.float64)
        for i, b in enumerate(blocks):
            s = np.ascontiguousarray(b.samples)
            keep.append(s)
            sp = specs[i]
            sp.samples = s.ctypes.data
            sp.n = s.size
            sp.dtype = _NP_TO_PT[s.dtype]
            sp.scale, sp.fs, sp.t0 = float(b.scale), float(b.fs), float(b.t0)
            bb = np.asarray(b.bounds, dtype=np.float64).reshape(-1)
            for j in range(10):
                sp.bounds[j] = float(bb[j])
            if self._dim == 7:
                ext[i] = bb[10:14]
            sp.pop, sp.gens = int(b.pop), int(b.gens)
            sp.F, sp.CR = float(b.F), float(b.CR)
            sp.seed, sp.block_id = int(b.de_seed), int(b.block_id)
        self._h = ctypes.c_void_p()
        if self._dim == 7:
            ctx._check(self._lib.pt_batch_create_full(ctx.handle, specs,
                                                      ext.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                                                      int(tier), int(group_ctas), ctypes.byref(self._h)))
        else:
            ctx._check(self._lib.pt_batch_create(ctx.handle, specs, n, int(tier), int(group_ctas),
                                                 ctypes.byref(self._h)))
        self.n = n

    def run(self) -> float:
        """Solve every block; returns the device time in ms."""
        self._ctx._check(self._lib.pt_batch_run(self._h))
        return self.info()["last_ms"]

    def results(self):
        """(params[n, 5] or [n, 7] for the full model, sse[n]) of the last run."""
        out = np.zeros((self.n, 8), dtype=np.float64)
        self._ctx._check(self._lib.pt_batch_results_full(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out[:, :self._dim].copy(), out[:, 7].copy()

    def info(self) -> dict:
        i = BatchInfo()
        self._ctx._check(self._lib.pt_batch_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if self._h:
            self._lib.pt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving and block-to-block tracking -----------------------------------------


class Request(ctypes.Structure):
    """Mirror of ``pt_request``."""
    _fields_ = [("block", BlockSpec), ("tier", ctypes.c_int), ("stream_id", ctypes.c_int), ("model", ctypes.c_int),
                ("ext_bounds", ctypes.c_double * 4)]


class Result(ctypes.Structure):
    """Mirror of ``pt_result``."""
    _fields_ = [("fit", Fit), ("status", ctypes.c_int), ("stream_id", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("ext_params", ctypes.c_double * 2)]


def _serve_protos(lib):
    if getattr(lib, "_serve_protos", False):
        return
    vp = ctypes.c_void_p
    lib.pt_serve_configure.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
    lib.pt_serve_configure.restype = ctypes.c_int
    lib.pt_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.pt_submit.restype = ctypes.c_int
    lib.pt_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    lib.pt_poll.restype = ctypes.c_int
    lib.pt_clock.argtypes = []
    lib.pt_clock.restype = ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lib.pt_warm_bounds.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, dp]
    lib.pt_warm_bounds.restype = ctypes.c_int
    lib.pt_continuity.argtypes = [dp, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
    lib.pt_continuity.restype = ctypes.c_int
    lib.pt_warm_bounds_full.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, dp]
    lib.pt_warm_bounds_full.restype = ctypes.c_int
    lib.pt_continuity_full.argtypes = [dp, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       dp, dp]
    lib.pt_continuity_full.restype = ctypes.c_int
    lib._serve_protos = True


def _dvec(a, n):
    v = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    assert v.size == n
    return v


PIPE_COS, PIPE_FFMA, PIPE_DFMA, PIPE_EX2 = 0, 1, 2, 3


def pipe_rate(device: int, kind: int, nffma: int = 0) -> dict:
    """pt_pipe_rate: a pipe microbenchmark on ``device`` (PIPE_COS with
    ``nffma`` FP32 FMAs per cosine, PIPE_FFMA, PIPE_DFMA, PIPE_EX2). Returns operations
    per SM clock per SM (clock64), per second over the GPU (CUDA events), and
    the SM clock in MHz those imply."""
    lib = load_library()
    if not hasattr(lib, "_pipe_proto"):
        dp = ctypes.POINTER(ctypes.c_double)
        lib.pt_pipe_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.pt_pipe_rate.restype = ctypes.c_int
        lib._pipe_proto = True
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.pt_pipe_rate(int(device), int(kind), int(nffma), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc != PT_OK:
        raise PhaseTrackError(rc, "pt_pipe_rate failed")
    return {"per_clk_sm": a.value, "per_s": b.value, "sm_mhz": c.value}


def warm_bounds(prev, dt: float, T_next: float, min_f0: float = 0.0, min_f1: float = 0.0, min_f2: float = 0.0):
    """pt_warm_bounds: running-time ranges of the next block from the previous fit (5 x 2)."""
    lib = load_library()
    _serve_protos(lib)
    p = _dvec(prev, 5)
    out = np.zeros(10, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.pt_warm_bounds(p.ctypes.data_as(dp), float(dt), float(T_next), float(min_f0), float(min_f1),
                            float(min_f2), out.ctypes.data_as(dp))
    if rc != PT_OK:
        raise PhaseTrackError(rc, "pt_warm_bounds")
    return out.reshape(5, 2)


def continuity(a, Ta: float, b, Tb: float, max_dphi: float, max_dfreq: float):
    """pt_continuity: (passed, |dphi| rad, |dF| rad/s) at the shared border of two blocks."""
    lib = load_library()
    _serve_protos(lib)
    av, bv = _dvec(a, 5), _dvec(b, 5)
    dphi, dfreq = ctypes.c_double(), ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.pt_continuity(av.ctypes.data_as(dp), float(Ta), bv.ctypes.data_as(dp), float(Tb), float(max_dphi),
                           float(max_dfreq), ctypes.byref(dphi), ctypes.byref(dfreq))
    if rc < 0:
        raise PhaseTrackError(rc, "pt_continuity")
    return bool(rc), dphi.value, dfreq.value


def warm_bounds_full(prev, dt: float, T_next: float, a1_range=None):
    """pt_warm_bounds_full: the full model's running-time ranges (7 x 2)."""
    lib = load_library()
    _serve_protos(lib)
    p = _dvec(prev, 7)
    out = np.zeros(14, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    a1 = None if a1_range is None else _dvec(a1_range, 2)
    rc = lib.pt_warm_bounds_full(p.ctypes.data_as(dp), float(dt), float(T_next),
                                 a1.ctypes.data_as(dp) if a1 is not None else None, out.ctypes.data_as(dp))
    if rc != PT_OK:
        raise PhaseTrackError(rc, "pt_warm_bounds_full")
    return out.reshape(7, 2)


def continuity_full(a, Ta: float, b, Tb: float, max_dphi: float, max_dfreq: float):
    """pt_continuity_full: as ``continuity`` for full-model fits (7 parameters)."""
    lib = load_library()
    _serve_protos(lib)
    av, bv = _dvec(a, 7), _dvec(b, 7)
    dphi, dfreq = ctypes.c_double(), ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.pt_continuity_full(av.ctypes.data_as(dp), float(Ta), bv.ctypes.data_as(dp), float(Tb),
                                float(max_dphi), float(max_dfreq), ctypes.byref(dphi), ctypes.byref(dfreq))
    if rc < 0:
        raise PhaseTrackError(rc, "pt_continuity_full")
    return bool(rc), dphi.value, dfreq.value


class Server:
    """The context's serving loop: ``submit`` queues a block (returns a ticket,
    or None when the queue is full), ``poll`` returns a result dict or None."""

    def __init__(self, ctx: Context, max_inflight: int = 4, ctas_per_request: int = 0, mem_budget_bytes: int = 0,
                 max_queued: int = 64):
        self._ctx = ctx
        self._lib = ctx._lib
        self._models = {}  # ticket -> model of the request
        _serve_protos(self._lib)
        ctx._check(self._lib.pt_serve_configure(ctx.handle, int(max_inflight), int(ctas_per_request),
                                                int(mem_budget_bytes), int(max_queued)))

    def submit(self, block, tier: int = TIER_F64, stream_id: int = 0, bounds=None):
        s = np.ascontiguousarray(block.samples)
        r = Request()
        sp = r.block
        sp.samples = s.ctypes.data
        sp.n = s.size
        sp.dtype = _NP_TO_PT[s.dtype]
        sp.scale, sp.fs, sp.t0 = float(block.scale), float(block.fs), float(block.t0)
        bb = np.asarray(block.bounds if bounds is None else bounds, dtype=np.float64).reshape(-1)
        if bb.size not in (10, 14):
            raise ValueError("submit: bounds must be 5 x 2 or 7 x 2")
        for j in range(10):
            sp.bounds[j] = float(bb[j])
        if bb.size == 14:  # the full model
            r.model = 1
            for j in range(4):
                r.ext_bounds[j] = float(bb[10 + j])
        sp.pop, sp.gens = int(block.pop), int(block.gens)
        sp.F, sp.CR = float(block.F), float(block.CR)
        sp.seed, sp.block_id = int(block.de_seed), int(block.block_id)
        r.tier, r.stream_id = int(tier), int(stream_id)
        t = ctypes.c_uint64()
        rc = self._lib.pt_submit(self._ctx.handle, ctypes.byref(r), ctypes.byref(t))
        if rc == PT_EAGAIN:
            return None
        self._ctx._check(rc)
        self._models[int(t.value)] = int(r.model)
        return int(t.value)

    def poll(self, ticket: int):
        r = Result()
        rc = self._lib.pt_poll(self._ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc == PT_PENDING:
            return None
        self._ctx._check(rc)
        params = list(r.fit.params)
        if self._models.pop(ticket, 0) == 1:
            params += list(r.ext_params)
        return {"params": np.array(params), "sse": r.fit.sse, "status": r.status,
                "stream_id": r.stream_id, "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}

    def clock(self) -> float:
        return float(self._lib.pt_clock())


class TrackConfig(ctypes.Structure):
    """Mirror of ``pt_track_config``."""
    _fields_ = [("pop", ctypes.c_int), ("gens", ctypes.c_int), ("F", ctypes.c_double), ("CR", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("tier", ctypes.c_int), ("max_dphi", ctypes.c_double),
                ("max_dfreq", ctypes.c_double), ("enlarge", ctypes.c_double), ("max_attempts", ctypes.c_int),
                ("count_interval", ctypes.c_double)]


class TrackResult(ctypes.Structure):
    """Mirror of ``pt_track_result``."""
    _fields_ = [("block_index", ctypes.c_int64), ("quality", ctypes.c_int), ("attempts", ctypes.c_int),
                ("params", ctypes.c_double * 7), ("sse", ctypes.c_double), ("dphi", ctypes.c_double),
                ("dfreq", ctypes.c_double), ("phi_left", ctypes.c_double), ("phi_right", ctypes.c_double),
                ("f_left", ctypes.c_double), ("f_right", ctypes.c_double), ("total_phase", ctypes.c_double),
                ("int_doppler", ctypes.c_double), ("interval_phase", ctypes.c_double),
                ("bounds", ctypes.c_double * 14)]


def _track_protos(lib):
    if getattr(lib, "_track_protos", False):
        return
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.pt_track_create.argtypes = [vp, ctypes.POINTER(TrackConfig), dp, ctypes.POINTER(vp)]
    lib.pt_track_create.restype = ctypes.c_int
    lib.pt_track_create_full.argtypes = [vp, ctypes.POINTER(TrackConfig), dp, ctypes.POINTER(vp)]
    lib.pt_track_create_full.restype = ctypes.c_int
    lib.pt_track_block.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(TrackResult)]
    lib.pt_track_block.restype = ctypes.c_int
    lib.pt_track_destroy.argtypes = [vp]
    lib.pt_track_destroy.restype = None
    lib._track_protos = True


class Tracker:
    """``pt_track``: block-to-block tracking of one stream on ``ctx`` (Sec. 3.1.4):
    warm-started ranges, the Eq. 3-1-2 continuity check, enlarge-and-retry up to
    ``max_attempts`` searches, and total phase / integration Doppler (Eq. 4-1-2).
    ``block`` returns a dict of the ``pt_track_result`` fields. With 7 x 2
    bounds the session fits the full model (``pt_track_create_full``) and
    ``params`` has 7 entries, else 5."""

    def __init__(self, ctx: Context, bounds, pop: int = 64, gens: int = 1250, F: float = 0.7, CR: float = 0.9,
                 seed: int = 0, tier: int = TIER_F64, max_dphi: float = 0.3, max_dfreq: float = 2 * np.pi * 1.0,
                 enlarge: float = 2.0, max_attempts: int = 3, count_interval: float = 0.0):
        self._ctx = ctx
        self._lib = ctx._lib
        _track_protos(self._lib)
        c = TrackConfig(int(pop), int(gens), float(F), float(CR), int(seed), int(tier), float(max_dphi),
                        float(max_dfreq), float(enlarge), int(max_attempts), float(count_interval))
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64).reshape(-1))
        if b.size not in (10, 14):
            raise ValueError("Tracker bounds: 5 or 7 (lo, hi) pairs")
        self._dim = b.size // 2
        create = self._lib.pt_track_create_full if self._dim == 7 else self._lib.pt_track_create
        h = ctypes.c_void_p()
        ctx._check(create(ctx.handle, ctypes.byref(c), b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          ctypes.byref(h)))
        self._h = h

    def block(self, samples, fs: float, scale: float = 1.0) -> dict:
        s = np.ascontiguousarray(samples)
        r = TrackResult()
        self._ctx._check(self._lib.pt_track_block(self._h, s.ctypes.data, s.size, _NP_TO_PT[s.dtype], float(scale),
                                                  float(fs), ctypes.byref(r)))
        out = {k: getattr(r, k) for k, _ in TrackResult._fields_}
        out["params"] = np.array(list(r.params)[:self._dim])
        out["bounds"] = np.array(list(r.bounds)[:2 * self._dim]).reshape(self._dim, 2)
        return out

    def close(self):
        if self._h:
            self._lib.pt_track_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
