"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws random numbers
(numpy PCG64) and sums random Fourier modes.  Every field it returns is a plain
float64 numpy array of shape (N, N, N) indexed [z, y, x].
"""
from __future__ import annotations

import math

import numpy as np

ADJOINT_SEED = 20911     # seed of the adjoint test directions
ENSEMBLE_SEED = 2505     # seed of the ensemble Re / M draws
ENSEMBLE_SIZES = (32, 48, 64, 96)
ENSEMBLE_PER_SIZE = 12
ENSEMBLE_RE = (400.0, 800.0, 1600.0, 3200.0)
ENSEMBLE_MACH = (0.1, 0.2)


def smooth_field(n: int, seed: int, n_modes: int = 8, kmax: int = 4,
                 length: float = 2.0 * math.pi) -> np.ndarray:
    """Sum of `n_modes` random real Fourier modes with integer wavevectors
    |k_i| <= kmax, Gaussian amplitudes and uniform phases, scaled to unit RMS.
    Periodic on [0, length)^3 and smooth (band-limited well below Nyquist for
    n >= 16)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.arange(n) * (length / n) * (2.0 * math.pi / length)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    f = np.zeros((n, n, n))
    for _ in range(n_modes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            k[0] = 1
        a = rng.normal()
        phase = rng.uniform(0.0, 2.0 * math.pi)
        f += a * np.cos(k[0] * x + k[1] * y + k[2] * z + phase)
    rms = math.sqrt(float(np.mean(f * f)))
    return f / rms if rms > 0 else f


def random_flow_fields(n: int, seed: int, amp_u: float = 1.0, amp_rho: float = 0.05,
                       amp_p: float = 0.2):
    """Smooth random (rho, u, v, w, p) fluctuations around rho = 1, zero mean
    velocity: returns (rho, u, v, w, dp) where the caller adds its own mean
    pressure. No symmetry of the TGV field survives, so indexing errors that a
    symmetric field would hide show up."""
    rho = 1.0 + amp_rho * smooth_field(n, seed * 7 + 1)
    u = amp_u * smooth_field(n, seed * 7 + 2)
    v = amp_u * smooth_field(n, seed * 7 + 3)
    w = amp_u * smooth_field(n, seed * 7 + 4)
    dp = amp_p * smooth_field(n, seed * 7 + 5)
    return rho, u, v, w, dp


def adjoint_directions(n: int, count: int = 16):
    """`count` seeded unit-RMS direction triples (for rho u, rho v, rho w)."""
    out = []
    for s in range(count):
        base = ADJOINT_SEED * 1000 + 3 * s
        out.append(np.stack([smooth_field(n, base + c) for c in range(3)]))
    return out


def ensemble_draws():
    """(n, Re, M) for the 48-instance ensemble: 12 each of 32^3, 48^3, 64^3, 96^3,
    Re from {400, 800, 1600, 3200} and M from {0.1, 0.2}, drawn in instance
    order from PCG64(2505)."""
    rng = np.random.Generator(np.random.PCG64(ENSEMBLE_SEED))
    out = []
    for n in ENSEMBLE_SIZES:
        for _ in range(ENSEMBLE_PER_SIZE):
            re = ENSEMBLE_RE[int(rng.integers(0, len(ENSEMBLE_RE)))]
            m = ENSEMBLE_MACH[int(rng.integers(0, len(ENSEMBLE_MACH)))]
            out.append((n, re, m))
    return out
