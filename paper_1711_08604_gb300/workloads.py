"""Seeded synthetic signals for Core AFD (arXiv:1711.08604).

This module only synthesises inputs: samples G(z_m) on the N points
z_m = exp(2 pi i m / N) and radial grids.  It holds none of the decomposition's
arithmetic (no inner products, selection or remainder update), so the CUDA path
and the CPU oracle can both be fed from it without sharing method code.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng``) with
seed = 1000 * workload number + item index, so every run sees the same inputs.
"Complex standard Gaussian" means (X + iY)/sqrt(2) with X, Y standard normal.

Workloads (sizes as in the benchmark definitions):

1. ``kernel_sum``  N=256, radii i/50 (M=50), K=10: G = sum_{j=1..5} w_j e_{b_j},
   b_j area-uniform in |b| <= 0.9, w_j complex standard Gaussian.  The
   normalised Szego kernel e_b(z) = sqrt(1-|b|^2)/(1 - conj(b) z) is the
   dictionary element of Sec. 2; here it only shapes the input.
2. ``tones``       N=4096, radii i/200 (M=200), K=50: 20 cosines with seeded
   integer frequencies in 1..500, amplitude 1/f, uniform phase, plus
   N(0, 0.01^2) noise; then the positive-frequency projection.
3. ``batch``       1024 signals, N uniform over {1024, 2048, 4096, 8192},
   radii i/100 (M=100), K=30: 5..40 tones per signal with frequencies below N/8.
4. ``serving``     Poisson arrivals at 2000/s for 10 s; N uniform over
   {512, ..., 16384}; radii i/128 (M=128); stop at delta <= 1e-4 or K=64;
   G = sum of 3..30 Szego kernels with |b| <= 0.95 plus complex noise 1e-3.
5. ``chirp``       N=65536, radii i/1000 (M=1000), K=100: a linear chirp over
   frequencies 10..8000 plus 50 tones (amplitude 0.5), projected.

Paper signals (Sec. 4.1): ``paper_f1`` (Case 1, a rational function in H^2)
and ``paper_f2`` (Case 2, sgn(sin t), projected onto positive frequencies).

Positive-frequency projection: keep DFT bins 0..N/2-1, zero bins N/2..N-1
(the Nyquist bin included), no doubling.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Signal", "sample_points", "szego_sum", "project_positive", "kernel_sum", "tones",
    "batch", "serving_requests", "chirp", "paper_f1", "paper_f2", "radii_linear",
    "radii_paper", "random_signal",
]


@dataclass
class Signal:
    """One decomposition request: samples, radial grid, step limit, stop tolerance."""
    G: np.ndarray          # complex128, N samples G(z_m)
    radii: np.ndarray      # float64, ascending, in [0, 1)
    K: int                 # maximum number of greedy steps
    tol: float = 0.0       # stop once delta <= tol (0: run all K steps)
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.G.size)

    @property
    def M(self) -> int:
        return int(self.radii.size)


def sample_points(N: int) -> np.ndarray:
    """z_m = exp(2 pi i m / N), m = 0..N-1."""
    t = 2.0 * np.pi * np.arange(N) / N
    return np.cos(t) + 1j * np.sin(t)


def radii_linear(M: int) -> np.ndarray:
    """r_i = i / M, i = 0..M-1."""
    return np.arange(M, dtype=np.float64) / M


def radii_paper() -> np.ndarray:
    """r = 0, 0.1, ..., 0.8 (the radii of the experiments of Sec. 4)."""
    return np.arange(9, dtype=np.float64) / 10.0


def _cgauss(rng, n) -> np.ndarray:
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2.0)


def _disc_uniform(rng, n, rmax) -> np.ndarray:
    rad = rmax * np.sqrt(rng.random(n))
    ang = 2.0 * np.pi * rng.random(n)
    return rad * (np.cos(ang) + 1j * np.sin(ang))


def szego_sum(N: int, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Samples of sum_j w_j sqrt(1-|b_j|^2) / (1 - conj(b_j) z) at z_m."""
    z = sample_points(N)
    G = np.zeros(N, dtype=np.complex128)
    for bj, wj in zip(np.atleast_1d(b), np.atleast_1d(w)):
        G += wj * np.sqrt(1.0 - abs(bj) ** 2) / (1.0 - np.conj(bj) * z)
    return G


def project_positive(x: np.ndarray) -> np.ndarray:
    """Keep DFT bins 0..N/2-1 of x, zero the rest (Nyquist included)."""
    X = np.fft.fft(np.asarray(x, dtype=np.complex128))
    X[x.size // 2:] = 0.0
    return np.fft.ifft(X)


def _tone_signal(rng, N: int, freqs: np.ndarray, amps: np.ndarray, noise: float) -> np.ndarray:
    t = 2.0 * np.pi * np.arange(N) / N
    phases = 2.0 * np.pi * rng.random(freqs.size)
    x = np.zeros(N)
    for f, a, p in zip(freqs, amps, phases):
        x += a * np.cos(f * t + p)
    if noise > 0.0:
        x += noise * rng.standard_normal(N)
    return project_positive(x)


def kernel_sum(item: int = 0, N: int = 256, M: int = 50, K: int = 10, n_kernels: int = 5,
               rmax: float = 0.9) -> Signal:
    """Workload 1: a sum of 5 seeded normalised Szego kernels."""
    rng = np.random.default_rng(1000 * 1 + item)
    b = _disc_uniform(rng, n_kernels, rmax)
    w = _cgauss(rng, n_kernels)
    return Signal(szego_sum(N, b, w), radii_linear(M), K, 0.0, {"workload": "kernel_sum", "b": b, "w": w})


def tones(item: int = 0, N: int = 4096, M: int = 200, K: int = 50, n_tones: int = 20,
          fmax: int = 500, noise: float = 0.01) -> Signal:
    """Workload 2: 20 seeded cosines (amplitude 1/f) plus noise, projected."""
    rng = np.random.default_rng(1000 * 2 + item)
    f = rng.choice(np.arange(1, fmax + 1), size=n_tones, replace=False)
    G = _tone_signal(rng, N, f, 1.0 / f, noise)
    return Signal(G, radii_linear(M), K, 0.0, {"workload": "tones", "freqs": f})


def batch(n_signals: int = 1024, Ns=(1024, 2048, 4096, 8192), M: int = 100, K: int = 30,
          seed_item: int = 0) -> list:
    """Workload 3: signals of uneven N, 5..40 tones each with frequencies below N/8."""
    out = []
    for i in range(n_signals):
        rng = np.random.default_rng(1000 * 3 + seed_item + i)
        N = int(rng.choice(np.asarray(Ns)))
        q = int(rng.integers(5, 41))
        f = rng.choice(np.arange(1, N // 8), size=q, replace=False)
        G = _tone_signal(rng, N, f, 1.0 / f, 0.01)
        out.append(Signal(G, radii_linear(M), K, 0.0, {"workload": "batch", "item": i}))
    return out


def serving_requests(rate: float = 2000.0, duration: float = 10.0,
                     Ns=(512, 1024, 2048, 4096, 8192, 16384), M: int = 128, K: int = 64,
                     tol: float = 1e-4, max_requests: int | None = None, seed_item: int = 0):
    """Workload 4: (arrival time in s, Signal) pairs of a seeded Poisson stream."""
    rng = np.random.default_rng(1000 * 4 + seed_item)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration or (max_requests is not None and len(reqs) >= max_requests):
            break
        i = len(reqs)
        r2 = np.random.default_rng(1000 * 4 + seed_item + 1 + i)
        N = int(r2.choice(np.asarray(Ns)))
        q = int(r2.integers(3, 31))
        b = _disc_uniform(r2, q, 0.95)
        w = _cgauss(r2, q)
        G = szego_sum(N, b, w) + 1e-3 * _cgauss(r2, N)
        reqs.append((t, Signal(G, radii_linear(M), K, tol, {"workload": "serving", "item": i})))
    return reqs


def chirp(item: int = 0, N: int = 65536, M: int = 1000, K: int = 100, n_tones: int = 50,
          f0: float = 10.0, f1: float = 8000.0, tone_amp: float = 0.5) -> Signal:
    """Workload 5: linear chirp over frequencies f0..f1 (cycles per circle) plus tones."""
    rng = np.random.default_rng(1000 * 5 + item)
    u = np.arange(N) / N
    x = np.cos(2.0 * np.pi * (f0 * u + (f1 - f0) * u * u / 2.0))
    t = 2.0 * np.pi * u
    f = rng.integers(1, int(f1) + 1, size=n_tones)
    ph = 2.0 * np.pi * rng.random(n_tones)
    for fq, p in zip(f, ph):
        x = x + tone_amp * np.cos(fq * t + p)
    return Signal(project_positive(x), radii_linear(M), K, 0.0, {"workload": "chirp"})


def paper_f1(N: int = 1024) -> np.ndarray:
    """Case 1 of Sec. 4.1: (0.0247 e^{3it} + 0.355 e^{2it}) / (1 - 0.3679 e^{it})."""
    z = sample_points(N)
    return (0.0247 * z ** 3 + 0.355 * z ** 2) / (1.0 - 0.3679 * z)


def paper_f2(N: int = 1024) -> np.ndarray:
    """Case 2 of Sec. 4.1: sgn(sin t) with sgn(0) = 0, projected onto positive frequencies."""
    t = 2.0 * np.pi * np.arange(N) / N
    s = np.sin(t)
    s[0] = 0.0
    if N % 2 == 0:
        s[N // 2] = 0.0
    return project_positive(np.sign(s))


def random_signal(N: int, seed: int) -> np.ndarray:
    """Complex standard Gaussian samples (tests of small cases)."""
    return _cgauss(np.random.default_rng(seed), N)


# ----------------------------------------------------- non-uniform samples --

def nonuniform_angles(N: int, seed: int, jitter: float = 0.45) -> np.ndarray:
    """N ascending angles in [0, 2 pi): 2 pi (m + jitter U_m) / N, U_m uniform
    in (-1, 1) (seeded), kept ascending by jitter < 0.5."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, N)
    t = 2.0 * np.pi * (np.arange(N) + 0.5 + jitter * u) / N
    return np.sort(np.mod(t, 2.0 * np.pi))


def trapezoid_weights(theta: np.ndarray) -> np.ndarray:
    """Quadrature weights of the normalised measure dt / 2 pi on the circle:
    half the arc to each neighbour, (theta_{m+1} - theta_{m-1}) / (4 pi),
    cyclically; they sum to 1."""
    t = np.asarray(theta, dtype=np.float64)
    nxt = np.roll(t, -1)
    nxt[-1] += 2.0 * np.pi
    prv = np.roll(t, 1)
    prv[0] -= 2.0 * np.pi
    return (nxt - prv) / (4.0 * np.pi)


def szego_sum_at(theta: np.ndarray, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_j w_j sqrt(1-|b_j|^2) / (1 - conj(b_j) z) at z = exp(i theta)."""
    z = np.exp(1j * np.asarray(theta, dtype=np.float64))
    G = np.zeros(z.size, dtype=np.complex128)
    for bj, wj in zip(np.atleast_1d(b), np.atleast_1d(w)):
        G += wj * np.sqrt(1.0 - abs(bj) ** 2) / (1.0 - np.conj(bj) * z)
    return G


@dataclass
class NonuniformSignal:
    theta: np.ndarray
    weights: np.ndarray
    G: np.ndarray
    radii: np.ndarray
    L: int
    K: int

    @property
    def N(self) -> int:  # samples
        return int(self.theta.size)

    @property
    def M(self) -> int:  # radii
        return int(self.radii.size)


def nonuniform(item: int = 0, N: int = 3000, L: int = 1024, M: int = 64, K: int = 12) -> NonuniformSignal:
    """Non-uniform sampling case: N jittered angles with trapezoid weights, a
    grid of L equispaced angles and M radii i/M; G = 3..12 Szego kernels with
    |b| <= 0.9 (area-uniform) and complex Gaussian weights, plus complex noise
    1e-3."""
    rng = np.random.default_rng(6000 + item)
    theta = nonuniform_angles(N, 6500 + item)
    q = int(rng.integers(3, 13))
    b = 0.9 * np.sqrt(rng.uniform(0, 1, q)) * np.exp(2j * np.pi * rng.uniform(0, 1, q))
    G = szego_sum_at(theta, b, _cgauss(rng, q)) + 1e-3 * _cgauss(rng, N)
    return NonuniformSignal(theta, trapezoid_weights(theta), G, radii_linear(M), L, K)
