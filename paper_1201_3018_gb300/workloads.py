"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only -- no step of the method.  The CUDA
path, the CPU oracle, the tests and the benchmark all draw their inputs here so
that every side sees the same numbers.

The paper's application data (the cover-song beat/chroma features of Section
IV.B and the MPEG-7 audio clips of Section IV.C) are not available, so the
marginals the paper reports stand in for them: zero-mean Laplacian audio
samples (Section IV.D, Fig. 4b), Gaussian and uniform test signals (Section
IV.A uses U[-128, 128]).  Every generator uses numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 12013018


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


@dataclasses.dataclass
class ConvCase:
    name: str
    s: np.ndarray          # FP32 input, length L
    k: np.ndarray          # FP32 kernel (or template for xcorr), length N
    Wblock: int
    xcorr: bool = False
    fft: bool = False
    snr_db: float | None = None   # per-block adaptive target
    Sq: int = 0                   # fixed quantiser (0 = none)
    Kq: int = 0


def single_conv(seed: int = SEED_BASE + 1, L: int = 65536, N: int = 64, Wblock: int = 1024) -> ConvCase:
    """Single convolution: N(0,1) input, U[-1,1] kernel, direct core."""
    g = rng(seed)
    s = _f32(g.standard_normal(L))
    k = _f32(g.uniform(-1.0, 1.0, N))
    return ConvCase("single_conv_L%d_N%d_W%d" % (L, N, Wblock), s, k, Wblock)


def matching_xcorr(seed: int = SEED_BASE + 2, L: int = 1 << 20, N: int = 4096, Wblock: int = 8192,
                   scale: float = 0.1, noise_var: float = 0.01, snr_db: float = 45.0) -> ConvCase:
    """Matching-shaped cross-correlation: a Laplacian(0, scale) signal and a
    template cut from it plus Gaussian noise of variance noise_var."""
    g = rng(seed)
    s = g.laplace(0.0, scale, L)
    a = int(g.integers(0, max(1, L - N)))
    t = s[a:a + N] + g.normal(0.0, math.sqrt(noise_var), N)
    return ConvCase("matching_xcorr_L%d_N%d_W%d" % (L, N, Wblock), _f32(s), _f32(t), Wblock,
                    xcorr=True, fft=True, snr_db=snr_db)


def uniform_e1(seed: int = SEED_BASE + 6, L: int = 8192 * 1024, N: int = 800, Wblock: int = 32 * 1024,
               amp: float = 128.0) -> ConvCase:
    """Section IV.A throughput-test shape: U[-amp, amp] signal and kernel."""
    g = rng(seed)
    s = _f32(g.uniform(-amp, amp, L))
    k = _f32(g.uniform(-amp, amp, N))
    return ConvCase("uniform_L%d_N%d_W%d" % (L, N, Wblock), s, k, Wblock)


@dataclasses.dataclass
class BatchCase:
    name: str
    signals: list
    kernels: list
    targets: list


def batched_uneven(seed: int = SEED_BASE + 3, count: int = 256, lmin_log2: float = 14.0,
                   lmax_log2: float = 20.0, taps=(256, 1024), targets=(30.0, 45.0, 60.0),
                   scale: float = 0.1) -> BatchCase:
    """Many signals of log-uniform length, Laplacian values, U[-1,1] kernels of
    alternating length, SNR targets drawn from a set."""
    g = rng(seed)
    sig, ker, tgt = [], [], []
    for i in range(count):
        L = int(2.0 ** g.uniform(lmin_log2, lmax_log2))
        sig.append(_f32(g.laplace(0.0, scale, L)))
        N = taps[i % len(taps)]
        ker.append(_f32(g.uniform(-1.0, 1.0, N)))
        tgt.append(float(targets[int(g.integers(0, len(targets)))]))
    return BatchCase("batched_uneven_%d" % count, sig, ker, tgt)


def windowed_sinc_bank(nfilt: int = 32, N: int = 1024, fs: float = 44100.0, f_lo: float = 50.0,
                       f_hi: float = 20000.0) -> np.ndarray:
    """Hann-windowed-sinc band-pass kernels with log-spaced band edges."""
    edges = np.geomspace(f_lo, f_hi, nfilt + 1)
    n = np.arange(N, dtype=np.float64) - (N - 1) / 2.0
    win = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(N) / (N - 1))
    bank = np.empty((nfilt, N), np.float64)
    for f in range(nfilt):
        a, b = edges[f] / fs, edges[f + 1] / fs
        h = 2.0 * b * np.sinc(2.0 * b * n) - 2.0 * a * np.sinc(2.0 * a * n)
        bank[f] = h * win
    return _f32(bank)


def filterbank(seed: int = SEED_BASE + 4, L: int = 1 << 22, nfilt: int = 32, N: int = 1024):
    g = rng(seed)
    return _f32(g.standard_normal(L)), windowed_sinc_bank(nfilt, N)


def random_signal(seed: int, L: int, dist: str = "normal", scale: float = 1.0) -> np.ndarray:
    g = rng(seed)
    if dist == "normal":
        x = g.standard_normal(L) * scale
    elif dist == "laplace":
        x = g.laplace(0.0, scale, L)
    elif dist == "uniform":
        x = g.uniform(-scale, scale, L)
    else:
        raise ValueError(dist)
    return _f32(x)


def serving_trace(seed: int = SEED_BASE + 5, rate_hz: float = 2000.0, duration_s: float = 1.0,
                  lmin_log2: float = 12.0, lmax_log2: float = 22.0, nmin: int = 64, nmax: int = 8192,
                  targets=(30.0, 45.0, 60.0), scale: float = 0.1):
    """Poisson arrivals of conv/xcorr requests: yields dicts with arrival time,
    op, lengths and target (signals are drawn lazily from the request seed)."""
    g = rng(seed)
    t = 0.0
    reqs = []
    while True:
        t += float(g.exponential(1.0 / rate_hz))
        if t > duration_s:
            break
        L = int(2.0 ** g.uniform(lmin_log2, lmax_log2))
        N = int(2.0 ** g.uniform(math.log2(nmin), math.log2(nmax)))
        N = max(1, min(N, L))
        reqs.append(dict(t=t, L=L, N=N, xcorr=bool(g.integers(0, 2)),
                         target=float(targets[int(g.integers(0, len(targets)))]),
                         seed=int(g.integers(0, 2 ** 31 - 1)), scale=scale))
    return reqs


def request_data(req) -> tuple:
    g = rng(req["seed"])
    return _f32(g.laplace(0.0, req["scale"], req["L"])), _f32(g.uniform(-1.0, 1.0, req["N"]))
