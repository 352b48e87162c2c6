"""Plain FP64 CPU oracle for the DE phase-tracking hot path (arxiv 1906.10598).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The CUDA
library never imports, links or calls it, and it never touches the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, FP64, libm ``cos``); this module
builds it with gcc and exposes numpy-friendly wrappers:

* ``sse`` / ``sse_many``  -- chi-square objective, Sec. 2.2 Eq. 2-2-4 with the
  model of Eq. 2-2-2 (c5 = 0) written in cycles.
* ``de_solve``            -- DE/rand/1/bin with the Table 3-1-1 controls.
* ``sse_full``, ``de_solve_full`` -- the full model of Eq. 2-2-2 (amplitude
  slope c5) with the phase to order n = 4 (Sec. 3.2), 7 parameters.
* ``de_textbook``         -- the same DE on sphere / Rosenbrock (self-check).
* ``de_trials``, ``pick3`` -- one generation's trial vectors and draws, and the
  index draw from given words (pins of the DE's one-step rules).
* ``philox4x32_10``       -- Salmon et al. SC'11 counter-based generator.
* ``theta_to_c``, ``c_phase``, ``c_freq``, ``c_total_phase`` -- Eq. 3-1-1 and
  Eq. 4-1-2 observables in the paper's c0..c3 coefficients.
* ``crb``                 -- Cramer-Rao bound from the exact Fisher matrix of
  the model (textbook estimation theory; the paper gives none).

Parity status: every function above is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, identities, brute force,
published known answers, the paper's Appendix 1 example).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

D = 5
# the full model of Sec. 2.2: (A, phi0, f0, f1, f2, A1, f3), amplitude slope
# c5 = A1 and the order-4 phase term f3 (cycles/s^4)
DF = 7


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oc_philox4x32_10.restype = None
        lib.oc_phase_cycles.argtypes = [dp, ctypes.c_double]
        lib.oc_phase_cycles.restype = ctypes.c_double
        lib.oc_model.argtypes = [dp, ctypes.c_double]
        lib.oc_model.restype = ctypes.c_double
        lib.oc_sse.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp]
        lib.oc_sse.restype = ctypes.c_double
        lib.oc_sse_many.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int64, dp,
                                    ctypes.c_int]
        lib.oc_sse_many.restype = None
        lib.oc_de_solve_block.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                          ctypes.c_uint32, dp, dp, dp, ctypes.c_int]
        lib.oc_de_solve_block.restype = ctypes.c_int
        lib.oc_de_solve_block_obj.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                              ctypes.c_uint32, ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int]
        lib.oc_de_textbook_strategy.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int, dp]
        lib.oc_de_textbook_strategy.restype = ctypes.c_int
        lib.oc_de_solve_block_obj.restype = ctypes.c_int
        for name in ("oc_cor", "oc_cor_objective"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp]
            fn.restype = ctypes.c_double
        lib.oc_cor_objective_many.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp,
                                              ctypes.c_int64, dp, ctypes.c_int]
        lib.oc_cor_objective_many.restype = None
        lib.oc_de_textbook.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, dp]
        lib.oc_de_textbook.restype = ctypes.c_int
        for name in ("oc_c_phase", "oc_c_freq", "oc_c_total_phase"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, ctypes.c_double]
            fn.restype = ctypes.c_double
        lib.oc_theta_to_c.argtypes = [dp, dp]
        lib.oc_theta_to_c.restype = None
        lib.oc_phase_cycles_full.argtypes = [dp, ctypes.c_double]
        lib.oc_phase_cycles_full.restype = ctypes.c_double
        lib.oc_model_full.argtypes = [dp, ctypes.c_double]
        lib.oc_model_full.restype = ctypes.c_double
        lib.oc_sse_full.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp]
        lib.oc_sse_full.restype = ctypes.c_double
        lib.oc_sse_full_many.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int64,
                                         dp, ctypes.c_int]
        lib.oc_sse_full_many.restype = None
        lib.oc_de_solve_block_full.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_uint64, ctypes.c_uint32, dp, dp, dp, ctypes.c_int]
        lib.oc_de_solve_block_full.restype = ctypes.c_int
        lib.oc_de_textbook_dim_strategy.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                                    dp]
        lib.oc_de_textbook_dim_strategy.restype = ctypes.c_int
        lib.oc_de_solve_block_full_strategy.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp,
                                                        ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, dp, dp, dp,
                                                        ctypes.c_int]
        lib.oc_de_solve_block_full_strategy.restype = ctypes.c_int
        lib.oc_pick3.argtypes = [ctypes.c_uint32, ctypes.c_uint32, u32p, u32p]
        lib.oc_pick3.restype = None
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oc_de_trials.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                     dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, u32p, u32p,
                                     u32p, ip, ip]
        lib.oc_de_trials.restype = ctypes.c_int
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 words for a 4-word counter, 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.oc_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def phase_cycles(theta, t: float) -> float:
    """p(t) = phi0/(2 pi) + f0 t + f1 t^2/2 + f2 t^3/6 (cycles)."""
    th = _f64(theta)
    return _load().oc_phase_cycles(_dptr(th), float(t))


def model(theta, t: float) -> float:
    th = _f64(theta)
    return _load().oc_model(_dptr(th), float(t))


def sse(samples, fs: float, t0: float, theta) -> float:
    """Eq. 2-2-4 objective of one candidate theta = (A, phi0, f0, f1, f2)."""
    s = _f64(samples)
    th = _f64(theta)
    return _load().oc_sse(_dptr(s), s.size, float(fs), float(t0), _dptr(th))


def sse_many(samples, fs: float, t0: float, cands, nthreads: int = 0) -> np.ndarray:
    """Eq. 2-2-4 objective for each row of ``cands`` (n x 5); OpenMP over rows."""
    s = _f64(samples)
    c = _f64(cands).reshape(-1, D)
    out = np.zeros(c.shape[0], dtype=np.float64)
    _load().oc_sse_many(_dptr(s), s.size, float(fs), float(t0), _dptr(c), c.shape[0], _dptr(out), int(nthreads))
    return out


def cor(samples, fs: float, t0: float, theta) -> float:
    """Eq. 2-2-5's cor: the unnormalised cross-correlation sum_i s_i m(t_i)."""
    s = _f64(samples)
    th = _f64(theta)
    return _load().oc_cor(_dptr(s), s.size, float(fs), float(t0), _dptr(th))


def cor_objective(samples, fs: float, t0: float, theta) -> float:
    """Eq. 2-2-5 objective 1 / (atan(cor) + pi/2) of one candidate."""
    s = _f64(samples)
    th = _f64(theta)
    return _load().oc_cor_objective(_dptr(s), s.size, float(fs), float(t0), _dptr(th))


def cor_objective_many(samples, fs: float, t0: float, cands, nthreads: int = 0) -> np.ndarray:
    s = _f64(samples)
    c = _f64(cands).reshape(-1, D)
    out = np.zeros(c.shape[0], dtype=np.float64)
    _load().oc_cor_objective_many(_dptr(s), s.size, float(fs), float(t0), _dptr(c), c.shape[0], _dptr(out),
                                  int(nthreads))
    return out


OBJECTIVES = {"chi2": 0, "cor": 1}
# DE strategies: the default rand/1/bin, and the paper's "3" and "6" (Table 3-1-1)
STRATEGIES = {"rand1bin": 0, "best1jitter": 3, "eitheror": 6}


def de_solve(samples, fs: float, t0: float, bounds, pop: int, gens: int, F: float, CR: float, seed: int,
             block_id: int = 0, nthreads: int = 0, return_population: bool = False, objective: str = "chi2",
             strategy: str = "rand1bin"):
    """DE/rand/1/bin fit of one block on the chi-square (Eq. 2-2-4) or the
    correlation (Eq. 2-2-5) objective. Returns (params[5], objective value)
    or, with ``return_population``, (params, value, population[pop,5],
    fitness[pop])."""
    s = _f64(samples)
    b = _f64(bounds).reshape(D, 2)
    out = np.zeros(D + 1, dtype=np.float64)
    popv = np.zeros((pop, D), dtype=np.float64)
    fit = np.zeros(pop, dtype=np.float64)
    rc = _load().oc_de_solve_block_obj(_dptr(s), s.size, float(fs), float(t0), _dptr(b), int(pop), int(gens),
                                       float(F), float(CR), ctypes.c_uint64(int(seed)),
                                       ctypes.c_uint32(int(block_id)), int(OBJECTIVES[objective]),
                                       int(STRATEGIES[strategy]), _dptr(out),
                                       _dptr(popv), _dptr(fit), int(nthreads))
    if rc != 0:
        raise ValueError("oracle de_solve: invalid arguments")
    if return_population:
        return out[:D].copy(), float(out[D]), popv, fit
    return out[:D].copy(), float(out[D])


def pick3(i: int, np_: int, words) -> np.ndarray:
    """The DE's index draw for individual i of a population of np_ from three
    given 32-bit words: r1, r2, r3 distinct and different from i."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    r = np.zeros(3, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    _load().oc_pick3(ctypes.c_uint32(int(i)), ctypes.c_uint32(int(np_)), w.ctypes.data_as(p), r.ctypes.data_as(p))
    return r


def de_trials(seed: int, block_id: int, gen: int, x, fx, bounds, F: float, CR: float,
              strategy: str = "rand1bin") -> dict:
    """One generation's trials (gen >= 1) from population x (pop x dim) with
    fitness fx: the trial vectors u, the drawn indices r (pop x 3), jrand, the
    crossover masks take (bit j: component j from the mutant), the either-or
    coin three_point and the previous generation's best index."""
    xx = _f64(x)
    pop, dim = xx.shape
    f = _f64(fx).reshape(pop)
    b = _f64(bounds).reshape(dim, 2)
    u = np.zeros((pop, dim), dtype=np.float64)
    r = np.zeros((pop, 3), dtype=np.uint32)
    jr = np.zeros(pop, dtype=np.uint32)
    tk = np.zeros(pop, dtype=np.uint32)
    tp = np.zeros(pop, dtype=np.int32)
    best = ctypes.c_int(-1)
    up = ctypes.POINTER(ctypes.c_uint32)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = _load().oc_de_trials(ctypes.c_uint64(int(seed)), ctypes.c_uint32(int(block_id)), ctypes.c_uint32(int(gen)),
                              int(pop), int(dim), _dptr(xx), _dptr(f), _dptr(b), float(F), float(CR),
                              int(STRATEGIES[strategy]), _dptr(u), r.ctypes.data_as(up), jr.ctypes.data_as(up),
                              tk.ctypes.data_as(up), tp.ctypes.data_as(ip), ctypes.byref(best))
    if rc != 0:
        raise ValueError("oracle de_trials: invalid arguments")
    return {"u": u, "r": r, "jrand": jr, "take": tk, "three_point": tp.astype(bool), "best": best.value}


def de_textbook(which: str, bounds, pop: int, gens: int, F: float, CR: float, seed: int,
                strategy: str = "rand1bin"):
    """The oracle's DE on a 5-D textbook function ('sphere' or 'rosenbrock')."""
    b = _f64(bounds).reshape(D, 2)
    out = np.zeros(D + 1, dtype=np.float64)
    rc = _load().oc_de_textbook_strategy(0 if which == "sphere" else 1, _dptr(b), int(pop), int(gens), float(F),
                                         float(CR), ctypes.c_uint64(int(seed)), int(STRATEGIES[strategy]),
                                         _dptr(out))
    if rc != 0:
        raise ValueError("oracle de_textbook: invalid arguments")
    return out[:D].copy(), float(out[D])


def phase_cycles_full(theta, t: float) -> float:
    """p(t) = phi0/(2 pi) + f0 t + f1 t^2/2 + f2 t^3/6 + f3 t^4/24 (cycles)."""
    th = _f64(theta)
    return _load().oc_phase_cycles_full(_dptr(th), float(t))


def model_full(theta, t: float) -> float:
    """(A + A1 t) cos(2 pi p(t)): Eq. 2-2-2 with c5 = A1, phase to order 4."""
    th = _f64(theta)
    return _load().oc_model_full(_dptr(th), float(t))


def sse_full(samples, fs: float, t0: float, theta) -> float:
    """Eq. 2-2-4 objective of one full-model candidate (7 parameters)."""
    s = _f64(samples)
    th = _f64(theta)
    return _load().oc_sse_full(_dptr(s), s.size, float(fs), float(t0), _dptr(th))


def sse_full_many(samples, fs: float, t0: float, cands, nthreads: int = 0) -> np.ndarray:
    s = _f64(samples)
    c = _f64(cands).reshape(-1, DF)
    out = np.zeros(c.shape[0], dtype=np.float64)
    _load().oc_sse_full_many(_dptr(s), s.size, float(fs), float(t0), _dptr(c), c.shape[0], _dptr(out),
                             int(nthreads))
    return out


def de_solve_full(samples, fs: float, t0: float, bounds, pop: int, gens: int, F: float, CR: float, seed: int,
                  block_id: int = 0, nthreads: int = 0, return_population: bool = False, strategy: str = "rand1bin"):
    """DE fit of the full model (7 parameters) on the chi-square (DE/rand/1/bin
    by default, or the strategies "3" and "6"). A parameter whose bounds are
    equal is held there (A1 = 0 or f3 = 0 gives the 6-parameter forms)."""
    s = _f64(samples)
    b = _f64(bounds).reshape(DF, 2)
    out = np.zeros(DF + 1, dtype=np.float64)
    popv = np.zeros((pop, DF), dtype=np.float64)
    fit = np.zeros(pop, dtype=np.float64)
    rc = _load().oc_de_solve_block_full_strategy(_dptr(s), s.size, float(fs), float(t0), _dptr(b), int(pop),
                                                 int(gens), float(F), float(CR), ctypes.c_uint64(int(seed)),
                                                 ctypes.c_uint32(int(block_id)), int(STRATEGIES[strategy]),
                                                 _dptr(out), _dptr(popv), _dptr(fit), int(nthreads))
    if rc != 0:
        raise ValueError("oracle de_solve_full: invalid arguments")
    if return_population:
        return out[:DF].copy(), float(out[DF]), popv, fit
    return out[:DF].copy(), float(out[DF])


def de_textbook_dim(which: str, bounds, pop: int, gens: int, F: float, CR: float, seed: int,
                    strategy: str = "rand1bin"):
    """The oracle's DE on a textbook function of len(bounds) parameters (5 or 7)."""
    b = _f64(bounds).reshape(-1, 2)
    dim = b.shape[0]
    out = np.zeros(dim + 1, dtype=np.float64)
    rc = _load().oc_de_textbook_dim_strategy(0 if which == "sphere" else 1, dim, _dptr(b), int(pop), int(gens),
                                             float(F), float(CR), ctypes.c_uint64(int(seed)),
                                             int(STRATEGIES[strategy]), _dptr(out))
    if rc != 0:
        raise ValueError("oracle de_textbook_dim: invalid arguments")
    return out[:dim].copy(), float(out[dim])


def theta_to_c(theta) -> np.ndarray:
    """(A, phi0, f0, f1, f2) -> paper coefficients (c0, c1, c2, c3, c4), Eq. 2-2-3."""
    th = _f64(theta)
    c = np.zeros(5, dtype=np.float64)
    _load().oc_theta_to_c(_dptr(th), _dptr(c))
    return c


def c_phase(c, t: float) -> float:
    """Eq. 3-1-1 phase (rad) from c0..c3."""
    cc = _f64(c)[:4].copy()
    return _load().oc_c_phase(_dptr(cc), float(t))


def c_freq(c, t: float) -> float:
    """Eq. 3-1-1 instantaneous frequency (rad/s) from c0..c3."""
    cc = _f64(c)[:4].copy()
    return _load().oc_c_freq(_dptr(cc), float(t))


def c_total_phase(c, T: float) -> float:
    """Eq. 4-1-2 for a single block of length T: phi(T/2) - phi(-T/2) (rad)."""
    cc = _f64(c)[:4].copy()
    return _load().oc_c_total_phase(_dptr(cc), float(T))


def crb(theta, n: int, fs: float, t0: float, sigma: float) -> np.ndarray:
    """Cramer-Rao standard deviations of (A, phi0, f0, f1, f2) for white
    Gaussian noise of standard deviation ``sigma``: the inverse of the Fisher
    matrix J = sigma^-2 sum_i grad m(t_i) grad m(t_i)^T at ``theta``, with
    m = A cos(phi0 + 2 pi (f0 t + f1 t^2/2 + f2 t^3/6)). Textbook result."""
    A, phi0, f0, f1, f2 = [float(v) for v in theta]
    t = t0 + np.arange(n, dtype=np.float64) / fs
    ph = phi0 + 2.0 * np.pi * (f0 * t + f1 * t * t / 2.0 + f2 * t ** 3 / 6.0)
    c, s = np.cos(ph), np.sin(ph)
    g = np.stack([c, -A * s, -A * s * 2 * np.pi * t, -A * s * np.pi * t * t, -A * s * np.pi * t ** 3 / 3.0])
    J = (g @ g.T) / (sigma * sigma)
    return np.sqrt(np.diag(np.linalg.inv(J)))


# ---------------------------------------------------------------------------
# Initial ranges of the first block from FFTs (Sec. 3.1.1): the frequency at
# the block centre from the spectrum of a small piece of data there, its rate
# by a central difference of three such frequencies, the amplitude from the
# spectral peak; ranges f0 and A +- 10 %, c3 in [-50, 50] rad/s^3, c5
# +- 0.2 c4 / T. Readings (the paper gives no more): pieces of Np samples
# (the largest power of two <= n/4, at most 8192), periodic Hann window,
# positive frequencies only (a real tone cannot tell f0 from -f0), peak bin
# refined by a parabola through the log magnitudes of the peak and its two
# neighbours, each piece's frequency taken at its sample Np/2 (the window's
# centre of symmetry), amplitude corrected by the window's response at the
# refined offset.

def seed_piece_len(n: int) -> int:
    """Np: the largest power of two <= n/4, at most 8192 (0 if n < 64)."""
    if n < 64:
        return 0
    return min(8192, 1 << int(np.floor(np.log2(n // 4))))


def seed_pieces(samples, piece_len: int = 0):
    """Refined peak of each of the three pieces: list of (start, bin, delta,
    |X[bin]|) with the centre piece second. Piece k starts at n//2 - Np/2 +
    (k - 1) Np."""
    x = _f64(samples)
    n = x.size
    Np = piece_len or seed_piece_len(n)
    if Np < 16 or Np & (Np - 1) or n // 2 - 3 * Np // 2 < 0 or n // 2 + 3 * Np // 2 > n:
        raise ValueError("seed: block too short for three pieces")
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(Np) / Np)
    out = []
    for k in range(3):
        s = n // 2 - Np // 2 + (k - 1) * Np
        X = np.fft.rfft(w * x[s:s + Np])
        mag = np.abs(X)
        kk = 1 + int(np.argmax(mag[1:Np // 2]))  # bins 1 .. Np/2 - 1, the first maximum
        a, b, g = np.log(mag[kk - 1]), np.log(mag[kk]), np.log(mag[kk + 1])
        den = a - 2.0 * b + g
        delta = 0.5 * (a - g) / den if den < 0.0 else 0.0
        out.append((s, kk, float(delta), float(mag[kk])))
    return out


def seed_bounds(samples, fs: float, t0: float, f0_rel: float = 0.1, piece_len: int = 0):
    """The FFT seed of Sec. 3.1.1 for the block t_i = t0 + i/fs: a dict with
    the estimates f0 (Hz at t = 0), f1 (Hz/s), A, the pieces' frequencies and
    bounds (7 x 2: A, phi0, f0, f1, f2, A1, f3; the first 5 rows are the cubic
    model's). f1's range is +- max(f0_rel |f1|, fs^2 / Np^2) (one bin over
    the pieces' spacing; the paper gives none), f3's is +- 192 / T^4 about 0
    (about +- pi rad at the block edge; the paper gives none)."""
    x = _f64(samples)
    n = x.size
    Np = piece_len or seed_piece_len(n)
    pieces = seed_pieces(x, Np)
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(Np) / Np)
    freqs, times = [], []
    for s, kk, delta, _ in pieces:
        freqs.append((kk + delta) * fs / Np)
        times.append(t0 + (s + Np // 2) / fs)
    f1 = (freqs[2] - freqs[0]) / (times[2] - times[0])
    f0 = freqs[1] - f1 * times[1]
    _, _, d1, m1 = pieces[1]
    resp = np.sinc(d1) / (1.0 - d1 * d1)  # the Hann window's response at the refined offset
    A = 2.0 * m1 / (np.sum(w) * resp)
    T = n / fs
    f2_max = 3.0 * 50.0 / np.pi  # c3 = pi f2 / 3 in [-50, 50] rad/s^3
    hw1 = max(f0_rel * abs(f1), fs * fs / (Np * Np))
    b = np.array([[(1.0 - f0_rel) * A, (1.0 + f0_rel) * A], [-np.pi, np.pi],
                  [f0 - f0_rel * abs(f0), f0 + f0_rel * abs(f0)], [f1 - hw1, f1 + hw1], [-f2_max, f2_max],
                  [-0.2 * A / T, 0.2 * A / T], [-192.0 / T ** 4, 192.0 / T ** 4]])
    return {"f0": float(f0), "f1": float(f1), "A": float(A), "piece_freqs": freqs, "piece_times": times,
            "piece_len": Np, "pieces": pieces, "bounds": b}
