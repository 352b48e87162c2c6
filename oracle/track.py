"""Block-to-block tracking of one stream, restated for the oracle (plain
Python over the oracle's DE fits).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module; it shares no
code with the CUDA library.

The paper's data process flow (Sec. 3.1.4) around the DE fit of each block:

* ranges (Sec. 3.1.1): the first block searches its initial ranges; every
  later block searches "running-time" ranges extrapolated from the last
  accepted fit to the new block's span. Reading used (the paper gives the
  frequency range as the previous fit's frequency from one border of the new
  block to the other): each range is the hull of the extrapolated quantity at
  the new block's left border, centre and right border, extended where needed
  to reach a minimum half-width about the centre value -- 2/T for the
  frequency, 4/T^2 for its rate, 24/T^3 for the cubic model's f2 (kept about
  the previous value) or for the full model's rate derivative, and 192/T^4
  for the full model's f3 (kept about the previous value); the amplitude
  range is +-10 % of the amplitude extrapolated to the new centre, phi0 the
  full circle, the full model's A1 its initial range. Parameters whose
  initial range is a point stay at that value.
* acceptance (Eq. 3-1-2): the fit passes when its phase and frequency at its
  left border agree with the reference fit's at that fit's right border
  within the thresholds (phase compared mod 2 pi). A block with no adjacent
  accepted predecessor (the first block, or the one after an abandoned
  block) is accepted unchecked.
* retry (Sec. 3.1.4): a failed search is repeated with the ranges of A, f0,
  f1, f2 (and f3) widened about their centres by the factor `enlarge` (an A
  range that would reach zero starts at 1e-3 of its top instead), phi0 and
  A1 unchanged, and the Philox key seed + (search - 1); after `max_attempts`
  failures the block is abandoned (quality 0): the adjacency is lost, the
  reference stays the last accepted fit (extrapolated across the gap), and
  the current count interval is discarded.
* quality index (Appendix 1's column, not defined by the paper): the number
  of the search that was accepted, 0 if abandoned.
* total phase (Eq. 4-1-2): phi(T/2) - phi(-T/2) = 2 pi (f0 T + f2 T^3 / 24)
  per accepted block (the even terms cancel), summed over a count interval;
  the interval ends at the first block that brings its length to at least
  count_interval seconds, whose record carries the interval's phase and the
  integration Doppler phase / length.
"""
from __future__ import annotations

import math

import numpy as np

from . import de_solve, de_solve_full

TWO_PI = 2.0 * math.pi


def _theta7(p) -> np.ndarray:
    """(A, phi0, f0, f1, f2[, A1, f3]) as 7 values (A1 = f3 = 0 for 5)."""
    q = np.zeros(7)
    p = np.asarray(p, dtype=np.float64)
    q[:p.size] = p
    return q


def phase_rad(p, t: float) -> float:
    """Eq. 3-1-1 phase at t (rad, not reduced) of a fit about its block centre."""
    A, phi0, f0, f1, f2, A1, f3 = _theta7(p)
    return phi0 + TWO_PI * (f0 * t + f1 * t ** 2 / 2 + f2 * t ** 3 / 6 + f3 * t ** 4 / 24)


def freq_rad(p, t: float) -> float:
    """Eq. 3-1-1 instantaneous frequency at t (rad/s)."""
    A, phi0, f0, f1, f2, A1, f3 = _theta7(p)
    return TWO_PI * (f0 + f1 * t + f2 * t ** 2 / 2 + f3 * t ** 3 / 6)


def continuity(ref, T_ref: float, fit, T: float):
    """Eq. 3-1-2 residuals (|dphi| mod 2 pi in [0, pi], |dF| in rad/s) between
    the reference fit's right border and the new fit's left border."""
    dphi = abs(math.remainder(phase_rad(ref, T_ref / 2) - phase_rad(fit, -T / 2), TWO_PI))
    dfreq = abs(freq_rad(ref, T_ref / 2) - freq_rad(fit, -T / 2))
    return dphi, dfreq


def _hull(fn, dt: float, T: float, min_half: float):
    """Hull of fn at the new block's borders and centre, extended to at least
    min_half either side of the centre value."""
    c = fn(dt)
    vals = (fn(dt - T / 2), fn(dt + T / 2), c, c - min_half, c + min_half)
    return min(vals), max(vals)


def running_ranges(prev, dt: float, T: float, dim: int, a1_range=None) -> np.ndarray:
    """Sec. 3.1.1 running-time ranges (dim x 2) of the block whose centre lies
    dt seconds after the centre of the fit `prev`, of length T."""
    A, phi0, f0, f1, f2, A1, f3 = _theta7(prev)
    r = np.zeros((dim, 2))
    r[1] = (-math.pi, math.pi)
    if dim == 5:
        amp = abs(A)
        r[2] = _hull(lambda t: f0 + f1 * t + f2 * t * t / 2, dt, T, 2 / T)
        r[3] = _hull(lambda t: f1 + f2 * t, dt, T, 4 / T ** 2)
        r[4] = (f2 - 24 / T ** 3, f2 + 24 / T ** 3)
    else:
        amp = abs(A + A1 * dt)
        r[2] = _hull(lambda t: f0 + f1 * t + f2 * t * t / 2 + f3 * t ** 3 / 6, dt, T, 2 / T)
        r[3] = _hull(lambda t: f1 + f2 * t + f3 * t * t / 2, dt, T, 4 / T ** 2)
        r[4] = _hull(lambda t: f2 + f3 * t, dt, T, 24 / T ** 3)
        r[5] = a1_range if a1_range is not None else (A1 - 0.2 * amp / T, A1 + 0.2 * amp / T)
        r[6] = (f3 - 192 / T ** 4, f3 + 192 / T ** 4)
    r[0] = (0.9 * amp, 1.1 * amp)
    return r


def hold_fixed(ranges: np.ndarray, init: np.ndarray) -> np.ndarray:
    """Parameters whose initial range is a point keep that value."""
    out = ranges.copy()
    for j in range(init.shape[0]):
        if init[j, 0] == init[j, 1]:
            out[j] = init[j, 0]
    return out


def widen(ranges: np.ndarray, factor: float) -> np.ndarray:
    """Sec. 3.1.4 range enlargement for a repeated search: A, f0, f1, f2 (and
    f3) about their centres by `factor`; phi0 and A1 unchanged; A kept positive."""
    out = ranges.copy()
    for j in (0, 2, 3, 4, 6):
        if j >= out.shape[0]:
            continue
        mid, half = (out[j, 0] + out[j, 1]) / 2, (out[j, 1] - out[j, 0]) / 2 * factor
        out[j] = (mid - half, mid + half)
    if out[0, 0] <= 0.0 < out[0, 1]:
        out[0, 0] = 1e-3 * out[0, 1]
    return out


def total_phase(p, T: float) -> float:
    """Eq. 4-1-2 term of one block: phi(T/2) - phi(-T/2) (rad)."""
    A, phi0, f0, f1, f2, A1, f3 = _theta7(p)
    return TWO_PI * (f0 * T + f2 * T ** 3 / 24)


class TrackSession:
    """One stream tracked block by block (Sec. 3.1.4), every fit by the
    oracle's DE (or by `solver(values, fs, t0, ranges, seed, block_id) ->
    (params, sse)` when given, e.g. to script the searches' outcomes)."""

    def __init__(self, bounds, pop: int = 64, gens: int = 1250, F: float = 0.7, CR: float = 0.9, seed: int = 0,
                 max_dphi: float = 0.3, max_dfreq: float = TWO_PI, enlarge: float = 2.0, max_attempts: int = 3,
                 count_interval: float = 0.0, solver=None, nthreads: int = 0):
        self.init = np.array(bounds, dtype=np.float64).reshape(-1, 2)
        self.dim = self.init.shape[0]
        if self.dim not in (5, 7):
            raise ValueError("5 or 7 (lo, hi) pairs")
        self.pop, self.gens, self.F, self.CR, self.seed = pop, gens, F, CR, seed
        self.max_dphi, self.max_dfreq = max_dphi, max_dfreq
        self.enlarge, self.max_attempts, self.count_interval = enlarge, max_attempts, count_interval
        self.solver = solver
        self.nthreads = nthreads
        self.index = 0
        self.ref = None          # last accepted fit
        self.ref_T = 0.0
        self.gap = 0.0           # seconds from the reference's right border to the end of the last block
        self.adjacent = False
        self.interval_phase, self.interval_T = 0.0, 0.0

    def _fit(self, values, fs, t0, ranges, seed, block_id):
        if self.solver is not None:
            return self.solver(values, fs, t0, ranges, seed, block_id)
        solve = de_solve if self.dim == 5 else de_solve_full
        return solve(values, fs, t0, ranges, self.pop, self.gens, self.F, self.CR, seed, block_id=block_id,
                     nthreads=self.nthreads)

    def first_ranges(self, T: float) -> np.ndarray:
        """The ranges of the next block's first search."""
        if self.ref is None:
            return self.init.copy()
        dt = self.ref_T / 2 + self.gap + T / 2
        a1 = tuple(self.init[5]) if self.dim == 7 else None
        return hold_fixed(running_ranges(self.ref, dt, T, self.dim, a1), self.init)

    def block(self, values, fs: float) -> dict:
        """Track the next block (physical sample values, centred time base)."""
        values = np.asarray(values, dtype=np.float64)
        n = values.size
        T = n / fs
        t0 = -(n - 1) / (2 * fs)
        ranges = self.first_ranges(T)
        searches = []
        quality = 0
        for a in range(1, self.max_attempts + 1):
            params, sse = self._fit(values, fs, t0, ranges, self.seed + a - 1, self.index)
            params = np.asarray(params, dtype=np.float64)
            if self.adjacent:
                dphi, dfreq = continuity(self.ref, self.ref_T, params, T)
                ok = dphi <= self.max_dphi and dfreq <= self.max_dfreq
            else:
                dphi = dfreq = math.nan
                ok = True
            searches.append({"ranges": ranges, "seed": self.seed + a - 1, "params": params, "sse": float(sse),
                             "dphi": dphi, "dfreq": dfreq, "accepted": ok})
            if ok:
                quality = a
                break
            if a < self.max_attempts:
                ranges = hold_fixed(widen(ranges, self.enlarge), self.init)
        last = searches[-1]
        p = last["params"]
        rec = {"block_index": self.index, "quality": quality, "attempts": len(searches), "params": p,
               "sse": last["sse"], "dphi": last["dphi"], "dfreq": last["dfreq"], "ranges": last["ranges"],
               "searches": searches, "phi_left": phase_rad(p, -T / 2) % TWO_PI,
               "phi_right": phase_rad(p, T / 2) % TWO_PI, "f_left": freq_rad(p, -T / 2),
               "f_right": freq_rad(p, T / 2), "total_phase": math.nan, "int_doppler": math.nan,
               "interval_phase": math.nan}
        self.index += 1
        if quality:
            rec["total_phase"] = total_phase(p, T)
            self.ref, self.ref_T, self.gap, self.adjacent = p, T, 0.0, True
            if self.count_interval > 0:
                self.interval_phase += rec["total_phase"]
                self.interval_T += T
                if self.interval_T >= self.count_interval * (1 - 1e-12):
                    rec["interval_phase"] = self.interval_phase
                    rec["int_doppler"] = self.interval_phase / self.interval_T
                    self.interval_phase, self.interval_T = 0.0, 0.0
        else:
            self.adjacent = False
            if self.ref is not None:
                self.gap += T
            self.interval_phase, self.interval_T = 0.0, 0.0
        return rec
