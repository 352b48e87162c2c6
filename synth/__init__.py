"""Seeded synthetic tracking blocks shaped like the paper's workloads.

This module only *generates data*: it holds neither the objective nor the DE
arithmetic, and both the CPU oracle and the CUDA path consume what it returns.
Randomness is numpy ``Generator(PCG64(seed))``; the DE's own random numbers are
drawn inside each implementation from Philox with the ``de_seed`` recorded here.

The paper's recordings (Mars Express, Chang'E-4 relay, Sec. 2.1 and Appendix 1)
are not available, so these blocks stand in for them: a real tone with a
cubic Taylor phase (Eq. 2-2-2, c5 = 0), white Gaussian noise at a stated
per-sample SNR = (A^2/2)/sigma^2, and 8/16-bit quantisation as produced by the
receiver recording modes of Table "PRSR data recording modes".

Workloads:
* ``single4096``   N = 4096 FP64 samples, fs = 1 kHz, pop 32, 200 generations.
* ``paper400k``    N = 400,000 int16 samples, fs = 10 kHz (40 s), pop 64,
                   1250 generations (~80,000 objective evaluations, the
                   400K-sample / 80,000-evaluation experiment of Sec. 1.3).
* ``precision``    the paper400k analog signal stored as int8 / int16 / FP16 /
                   FP32.
* ``batch``        256 blocks, N log-uniform in [5e4, 1e6], fs log-uniform in
                   [1, 50] kHz, pop uniform in 32..128, G = ceil(80000/pop).
* ``stream``       continuous-phase station streams for the serving loop.
* ``perigee400k``  the paper400k shape for the full model (amplitude slope
                   and quartic phase term, 7 parameters).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# sample storage codes (the C ABI uses the same numbering)
I8, I16, F16, F32, F64 = 0, 1, 2, 3, 4
STORAGE_NAMES = {"i8": I8, "i16": I16, "f16": F16, "f32": F32, "f64": F64}


@dataclasses.dataclass
class Block:
    samples: np.ndarray          # stored samples (dtype per ``dtype`` code)
    dtype: int                   # I8/I16/F16/F32/F64
    scale: float                 # physical value = scale * stored value
    fs: float                    # sampling rate, Hz
    t0: float                    # time of sample 0 (s); centred blocks use -(N-1)/(2 fs)
    truth: np.ndarray            # (A, phi0, f0, f1, f2) [+ (A1, f3) for the full model]
    sigma: float                 # noise standard deviation
    snr_db: float
    bounds: np.ndarray           # (5, 2) lo, hi  [(7, 2) for the full model]
    pop: int = 64
    gens: int = 1250
    F: float = 0.7
    CR: float = 0.9
    de_seed: int = 0
    block_id: int = 0
    noise: Optional[np.ndarray] = None   # the noise realisation (float64), for identities in tests

    @property
    def n(self) -> int:
        return int(self.samples.size)

    @property
    def T(self) -> float:
        return self.n / self.fs

    def values(self) -> np.ndarray:
        """Physical sample values in float64 (scale * stored)."""
        return self.samples.astype(np.float64) * self.scale

    def sample_evals(self) -> int:
        """Objective sample-evaluations of one DE solve: N * pop * (gens + 1)."""
        return self.n * self.pop * (self.gens + 1)


def centred_t0(n: int, fs: float) -> float:
    return -(n - 1) / (2.0 * fs)


def clean_tone(truth, n: int, fs: float, t0: float) -> np.ndarray:
    """Noise-free A cos(phi0 + 2 pi (f0 t + f1 t^2/2 + f2 t^3/6)) at t_i = t0 + i/fs."""
    A, phi0, f0, f1, f2 = [float(v) for v in truth]
    t = t0 + np.arange(n, dtype=np.float64) / fs
    return A * np.cos(phi0 + 2.0 * np.pi * (f0 * t + f1 * t * t / 2.0 + f2 * t ** 3 / 6.0))


def quantise(x: np.ndarray, full_scale: float, storage: int):
    """Store float64 values ``x`` in ``storage``; returns (stored, scale).

    int16: q = clamp(round_half_even(x / d), +-32767), d = full_scale / 30000
    int8:  q = clamp(round_half_even(x / d), +-127),   d = full_scale / 120
    fp16:  x / full_scale rounded to binary16, scale = full_scale
    fp32 / fp64: x itself, scale 1.
    """
    if storage == I16:
        d = full_scale / 30000.0
        return np.clip(np.rint(x / d), -32767, 32767).astype(np.int16), d
    if storage == I8:
        d = full_scale / 120.0
        return np.clip(np.rint(x / d), -127, 127).astype(np.int8), d
    if storage == F16:
        return (x / full_scale).astype(np.float16), float(full_scale)
    if storage == F32:
        return x.astype(np.float32), 1.0
    if storage == F64:
        return x.astype(np.float64), 1.0
    raise ValueError(f"unknown storage {storage}")


def _window(rng, truth_v: float, half_width: float):
    """[lo, hi] of width 2*half_width whose centre is offset from the truth by
    U(-1/2, 1/2) * half_width, so the truth is never the exact centre."""
    c = truth_v + rng.uniform(-0.5, 0.5) * half_width
    return c - half_width, c + half_width


def _sigma_for(A: float, snr_db: float) -> float:
    return math.sqrt(A * A / 2.0 / (10.0 ** (snr_db / 10.0)))


def single4096(seed: int = 0, n: int = 4096, fs: float = 1000.0, snr_db: float = 20.0) -> Block:
    """N = 4096 FP64 samples at 1 kHz, A = 1, phi0 ~ U(-pi, pi), f0 ~ U(-100, 100) Hz,
    f1 ~ U(-1, 1) Hz/s, f2 = 0, SNR 20 dB; bounds +-20% around the truth with floors
    (A 0.1, f0 1 Hz, f1 0.1 Hz/s, f2 0.01 Hz/s^2), phi0 over the full circle."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = 1.0
    truth = np.array([A, rng.uniform(-math.pi, math.pi), rng.uniform(-100, 100), rng.uniform(-1, 1), 0.0])
    sigma = _sigma_for(A, snr_db)
    t0 = centred_t0(n, fs)
    noise = rng.normal(0.0, sigma, n)
    x = clean_tone(truth, n, fs, t0) + noise
    floors = {0: 0.1, 2: 1.0, 3: 0.1, 4: 0.01}
    bounds = np.zeros((5, 2))
    bounds[1] = (-math.pi, math.pi)
    for j, fl in floors.items():
        bounds[j] = _window(rng, truth[j], max(0.2 * abs(truth[j]), fl))
    stored, scale = quantise(x, 1.0, F64)
    return Block(stored, F64, scale, fs, t0, truth, sigma, snr_db, bounds, pop=32, gens=200, F=0.7, CR=0.9,
                 de_seed=0, block_id=0, noise=noise)


def paper_bounds(rng, truth, T: float) -> np.ndarray:
    """FFT-seeded style windows: f0 +- 2/T, f1 +- 4/T^2, f2 +- 24/T^3 (each about
    +-pi rad of phase at the block edge), A +- 20%, phi0 over the full circle."""
    b = np.zeros((5, 2))
    b[0] = _window(rng, truth[0], 0.2 * truth[0])
    b[1] = (-math.pi, math.pi)
    b[2] = _window(rng, truth[2], 2.0 / T)
    b[3] = _window(rng, truth[3], 4.0 / T ** 2)
    b[4] = _window(rng, truth[4], 24.0 / T ** 3)
    return b


def _analog(seed: int, n: int, fs: float, f0_max: float, f1_max: float, f2_max: float, snr_range=(0.0, 30.0)):
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.uniform(0.5, 2.0)
    truth = np.array([A, rng.uniform(-math.pi, math.pi), rng.uniform(-f0_max, f0_max),
                      rng.uniform(-f1_max, f1_max), rng.uniform(-f2_max, f2_max)])
    snr_db = rng.uniform(*snr_range)
    sigma = _sigma_for(A, snr_db)
    t0 = centred_t0(n, fs)
    noise = rng.normal(0.0, sigma, n)
    x = clean_tone(truth, n, fs, t0) + noise
    bounds = paper_bounds(rng, truth, n / fs)
    return rng, truth, snr_db, sigma, t0, noise, x, bounds


def paper400k(seed: int = 0, n: int = 400_000, fs: float = 10_000.0, storage: int = I16, pop: int = 64,
              gens: int = 1250) -> Block:
    """Paper-size block: N = 400,000 samples at 10 kHz (40 s), int16; phi0 ~ U(-pi, pi),
    f0 ~ U(-2, 2) kHz, f1 ~ U(-5, 5) Hz/s, f2 ~ U(-0.05, 0.05) Hz/s^2, A ~ U(0.5, 2),
    SNR ~ U(0, 30) dB; pop 64, 1250 generations (64 * 1251 = 80,064 evaluations)."""
    _, truth, snr_db, sigma, t0, noise, x, bounds = _analog(seed, n, fs, 2000.0, 5.0, 0.05)
    stored, scale = quantise(x, truth[0] + 6.0 * sigma, storage)
    return Block(stored, storage, scale, fs, t0, truth, sigma, snr_db, bounds, pop=pop, gens=gens, F=0.7, CR=0.9,
                 de_seed=seed, block_id=0, noise=noise)


def precision(seed: int, storage: int, n: int = 400_000, fs: float = 10_000.0, gens: int = 1250) -> Block:
    """The paper400k analog signal of ``seed`` stored as ``storage`` (precision sweep)."""
    return paper400k(seed, n=n, fs=fs, storage=storage, gens=gens)


def clean_tone_full(truth, n: int, fs: float, t0: float) -> np.ndarray:
    """Noise-free (A + A1 t) cos(phi0 + 2 pi (f0 t + f1 t^2/2 + f2 t^3/6 + f3 t^4/24))
    for truth = (A, phi0, f0, f1, f2, A1, f3)."""
    A, phi0, f0, f1, f2, A1, f3 = [float(v) for v in truth]
    t = t0 + np.arange(n, dtype=np.float64) / fs
    return (A + A1 * t) * np.cos(phi0 + 2.0 * np.pi * (f0 * t + f1 * t * t / 2.0 + f2 * t ** 3 / 6.0
                                                       + f3 * t ** 4 / 24.0))


def perigee400k(seed: int = 0, n: int = 400_000, fs: float = 10_000.0, storage: int = I16, pop: int = 64,
                gens: int = 1250, snr_range=(10.0, 30.0)) -> Block:
    """Paper-size block of a high-dynamics arc (near perigee, where the paper
    takes the phase to order n = 4): N = 400,000 samples at 10 kHz, int16;
    the paper400k ranges for A, phi0, f0, f1, f2, plus an amplitude slope
    A1 ~ U(-0.1, 0.1) A / T and a quartic term f3 ~ U(-5e-4, 5e-4) cycles/s^4
    (a fourth phase derivative up to ~3e-3 rad/s^4, the order of the perigee
    figure of Sec. 3.2). truth and bounds have 7 rows (A, phi0, f0, f1, f2, A1,
    f3); A1's range is the paper's +-0.2 A / T, f3's window is +-192 / T^4
    (about +-pi rad at the block edge) around the truth, offset like the
    others."""
    rng = np.random.Generator(np.random.PCG64(seed + 7_000_003))
    T = n / fs
    A = rng.uniform(0.5, 2.0)
    truth = np.array([A, rng.uniform(-math.pi, math.pi), rng.uniform(-2000.0, 2000.0), rng.uniform(-5.0, 5.0),
                      rng.uniform(-0.05, 0.05), rng.uniform(-0.1, 0.1) * A / T, rng.uniform(-5e-4, 5e-4)])
    snr_db = rng.uniform(*snr_range)
    sigma = _sigma_for(A, snr_db)
    t0 = centred_t0(n, fs)
    noise = rng.normal(0.0, sigma, n)
    x = clean_tone_full(truth, n, fs, t0) + noise
    b5 = paper_bounds(rng, truth[:5], T)
    bounds = np.zeros((7, 2))
    bounds[:5] = b5
    bounds[5] = (-0.2 * b5[0, 1] / T, 0.2 * b5[0, 1] / T)
    bounds[6] = _window(rng, truth[6], 192.0 / T ** 4)
    peak = truth[0] + abs(truth[5]) * T / 2
    stored, scale = quantise(x, peak + 6.0 * sigma, storage)
    return Block(stored, storage, scale, fs, t0, truth, sigma, snr_db, bounds, pop=pop, gens=gens, F=0.7, CR=0.9,
                 de_seed=seed, block_id=0, noise=noise)


def batch(seed: int = 0, nblocks: int = 256, n_lo: int = 50_000, n_hi: int = 1_000_000, fs_lo: float = 1_000.0,
          fs_hi: float = 50_000.0, evals: int = 80_000) -> List[Block]:
    """Independent blocks of uneven length: N log-uniform in [n_lo, n_hi], fs log-uniform in
    [fs_lo, fs_hi], int16, pop uniform in 32..128, G = ceil(evals / pop). Chirp ranges are
    limited so the frequency excursion over a block stays well inside Nyquist."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(nblocks):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        fs = float(math.exp(rng.uniform(math.log(fs_lo), math.log(fs_hi))))
        T = n / fs
        f1_max = min(5.0, 0.1 * fs / T)
        f2_max = min(0.05, 0.4 * fs / T ** 2)
        sub = int(rng.integers(0, 2 ** 31))
        _, truth, snr_db, sigma, t0, noise, x, bounds = _analog(sub, n, fs, 0.4 * fs, f1_max, f2_max)
        stored, scale = quantise(x, truth[0] + 6.0 * sigma, I16)
        pop = int(rng.integers(32, 129))
        gens = int(math.ceil(evals / pop))
        out.append(Block(stored, I16, scale, fs, t0, truth, sigma, snr_db, bounds, pop=pop, gens=gens, F=0.7,
                         CR=0.9, de_seed=seed * 1000 + b, block_id=b, noise=None))
    return out


def batch_full(seed: int = 0, nblocks: int = 256, n_lo: int = 50_000, n_hi: int = 1_000_000, fs_lo: float = 1_000.0,
               fs_hi: float = 50_000.0, evals: int = 80_000) -> List[Block]:
    """The `batch` workload for the full model: the same block lengths, rates and
    populations, each tone with an amplitude slope A1 ~ U(-0.1, 0.1) A / T and a
    quartic term f3 ~ U(-1, 1) f3_max, f3_max = min(5e-4, 2.4 fs / T^3) cycles/s^4
    (the quartic's frequency excursion over the block stays within 5 % of fs);
    7 x 2 bounds: the `paper400k` windows, A1 over +-0.2 A / T, f3 +- 192 / T^4."""
    rng = np.random.Generator(np.random.PCG64(seed + 5_000_011))
    out = []
    for b in range(nblocks):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        fs = float(math.exp(rng.uniform(math.log(fs_lo), math.log(fs_hi))))
        T = n / fs
        f1_max = min(5.0, 0.1 * fs / T)
        f2_max = min(0.05, 0.4 * fs / T ** 2)
        f3_max = min(5e-4, 2.4 * fs / T ** 3)
        A = rng.uniform(0.5, 2.0)
        truth = np.array([A, rng.uniform(-math.pi, math.pi), rng.uniform(-0.4 * fs, 0.4 * fs),
                          rng.uniform(-f1_max, f1_max), rng.uniform(-f2_max, f2_max),
                          rng.uniform(-0.1, 0.1) * A / T, rng.uniform(-f3_max, f3_max)])
        snr_db = rng.uniform(0.0, 30.0)
        sigma = _sigma_for(A, snr_db)
        t0 = centred_t0(n, fs)
        x = clean_tone_full(truth, n, fs, t0) + rng.normal(0.0, sigma, n)
        bounds = np.zeros((7, 2))
        bounds[:5] = paper_bounds(rng, truth[:5], T)
        bounds[5] = (-0.2 * bounds[0, 1] / T, 0.2 * bounds[0, 1] / T)
        bounds[6] = _window(rng, truth[6], 192.0 / T ** 4)
        stored, scale = quantise(x, A * 1.1 + 6.0 * sigma, I16)
        pop = int(rng.integers(32, 129))
        gens = int(math.ceil(evals / pop))
        out.append(Block(stored, I16, scale, fs, t0, truth, sigma, snr_db, bounds, pop=pop, gens=gens, F=0.7,
                         CR=0.9, de_seed=seed * 1000 + b, block_id=b, noise=None))
    return out


@dataclasses.dataclass
class StreamSpec:
    """One simulated station stream with a continuous phase
    phi(t) = phi0 + 2 pi (F0 t + F1 t^2/2 + F2 t^3/6 + F3 t^4/24 + a sin(2 pi t / P))
    and amplitude A + A1 t (A1 = 0 unless set)."""
    stream_id: int
    fs: float
    block_s: float
    A: float
    snr_db: float
    phi0: float
    F0: float
    F1: float
    F2: float
    F3: float
    dop_a: float
    dop_p: float
    seed: int
    A1: float = 0.0


def make_streams(seed: int = 0, fs_list=(10_000.0, 20_000.0, 35_000.0, 50_000.0), block_range=(1.0, 10.0)):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k, fs in enumerate(fs_list):
        out.append(StreamSpec(k, float(fs), float(rng.uniform(*block_range)), float(rng.uniform(0.5, 2.0)),
                              float(rng.uniform(15.0, 30.0)), float(rng.uniform(-math.pi, math.pi)),
                              float(rng.uniform(-0.3, 0.3) * fs), float(rng.uniform(-5, 5)),
                              float(rng.uniform(-0.05, 0.05)), float(rng.uniform(-1e-4, 1e-4)),
                              float(rng.uniform(0.0, 0.2)), float(rng.uniform(200.0, 600.0)),
                              int(rng.integers(0, 2 ** 31))))
    return out


def stream_phase_cycles(spec: StreamSpec, t: np.ndarray) -> np.ndarray:
    return (spec.phi0 / (2 * math.pi) + spec.F0 * t + spec.F1 * t * t / 2 + spec.F2 * t ** 3 / 6
            + spec.F3 * t ** 4 / 24 + spec.dop_a * np.sin(2 * math.pi * t / spec.dop_p))


def stream_taylor_truth(spec: StreamSpec, tc: float) -> np.ndarray:
    """(A, phi0, f0, f1, f2) of the stream re-centred at time tc (Taylor coefficients
    of the continuous phase, Eq. 2-2-3); the quartic and sinusoid make the cubic model
    a truncation, bounded by Eq. 3-2-2."""
    w = 2 * math.pi / spec.dop_p
    a = spec.dop_a
    p0 = float(stream_phase_cycles(spec, np.array([tc]))[0])
    p1 = spec.F0 + spec.F1 * tc + spec.F2 * tc ** 2 / 2 + spec.F3 * tc ** 3 / 6 + a * w * math.cos(w * tc)
    p2 = spec.F1 + spec.F2 * tc + spec.F3 * tc ** 2 / 2 - a * w * w * math.sin(w * tc)
    p3 = spec.F2 + spec.F3 * tc - a * w ** 3 * math.cos(w * tc)
    ph = (p0 - math.floor(p0 + 0.5)) * 2 * math.pi
    return np.array([spec.A, ph, p1, p2, p3])


def stream_taylor_truth_full(spec: StreamSpec, tc: float) -> np.ndarray:
    """The full model's truth (A, phi0, f0, f1, f2, A1, f3) of the stream
    re-centred at tc: the cubic truth, the amplitude slope, and the fourth
    derivative of the phase; the sinusoid leaves an order-5 remainder."""
    w = 2 * math.pi / spec.dop_p
    t = stream_taylor_truth(spec, tc)
    p4 = spec.F3 + spec.dop_a * w ** 4 * math.sin(w * tc)
    return np.array([spec.A + spec.A1 * tc, t[1], t[2], t[3], t[4], spec.A1, p4])


def perigee_stream(seed: int = 0, fs: float = 2000.0, block_s: float = 10.0, snr_db: float = 25.0) -> StreamSpec:
    """A high-dynamics stream for the full model: a quartic phase whose
    t^4 term moves a 10 s block's edge phase by a few tenths of a radian
    (F3 ~ 2e-3 cycles/s^4, fourth derivative ~1e-2 rad/s^4), an amplitude
    slope of ~0.5 %/s, no sinusoid (the block truth is exact)."""
    rng = np.random.Generator(np.random.PCG64(seed + 9_000_011))
    return StreamSpec(0, float(fs), float(block_s), float(rng.uniform(0.8, 1.2)), float(snr_db),
                      float(rng.uniform(-math.pi, math.pi)), float(rng.uniform(-0.2, 0.2) * fs),
                      float(rng.uniform(-2, 2)), float(rng.uniform(-0.05, 0.05)),
                      float(rng.choice([-1.0, 1.0]) * rng.uniform(1.5e-3, 2.5e-3)), 0.0, 400.0,
                      int(rng.integers(0, 2 ** 31)), A1=float(rng.uniform(0.003, 0.006)))


def stream_block(spec: StreamSpec, index: int) -> Block:
    """Block ``index`` of a stream: samples over [index*T, (index+1)*T) stored int16,
    time origin at the block centre; bounds are the paper400k windows around the
    re-centred truth (the serving loop replaces them by warm-start windows)."""
    n = int(round(spec.block_s * spec.fs))
    fs = spec.fs
    start = index * n
    tc = (start + (n - 1) / 2.0) / fs
    t_abs = (start + np.arange(n, dtype=np.float64)) / fs
    rng = np.random.Generator(np.random.PCG64(spec.seed * 100_003 + index))
    sigma = _sigma_for(spec.A, spec.snr_db)
    noise = rng.normal(0.0, sigma, n)
    amp = spec.A + spec.A1 * t_abs if spec.A1 else spec.A
    x = amp * np.cos(2 * math.pi * stream_phase_cycles(spec, t_abs)) + noise
    truth = stream_taylor_truth(spec, tc)
    stored, scale = quantise(x, float(np.max(np.abs(amp))) + 6.0 * sigma, I16)
    bounds = paper_bounds(rng, truth, n / fs)
    return Block(stored, I16, scale, fs, centred_t0(n, fs), truth, sigma, spec.snr_db, bounds, pop=64,
                 gens=max(200, int(math.ceil(80_000 / 64))), F=0.7, CR=0.9, de_seed=spec.seed + index,
                 block_id=spec.stream_id * 1_000_000 + index, noise=noise)
