"""Pins of the oracle's stencils and time integrator (CPU only).

The 4th-order central differences of Sec. 2.3.1 are pinned by their Fourier
symbols (closed forms) and by numpy's FFT; the low-storage RK3 of Sec. 3.1
by its stability polynomial and its order of accuracy.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _plane_wave(n, k, axis):
    h = 2 * math.pi / n
    c = torch.arange(n, dtype=torch.float64) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    coord = (x, y, z)[axis]
    return torch.exp(1j * k * coord.to(torch.complex128)), h


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_first_derivative_symbol(axis):
    n = 16
    for k in range(0, n // 2 + 1):
        f, h = _plane_wave(n, k, axis)
        sym = 1j * (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h)
        g = oracle.d1(f, axis, h)
        assert torch.allclose(g, sym * f, atol=1e-12, rtol=0), (axis, k)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_second_derivative_symbol(axis):
    n = 16
    for k in range(0, n // 2 + 1):
        f, h = _plane_wave(n, k, axis)
        sym = -(30 - 32 * math.cos(k * h) + 2 * math.cos(2 * k * h)) / (12 * h * h)
        g = oracle.d2(f, axis, h)
        assert torch.allclose(g, sym * f, atol=1e-11, rtol=0), (axis, k)


def test_stencils_match_fft_on_random_field():
    rng = np.random.Generator(np.random.PCG64(7))
    n = 12
    h = 2 * math.pi / n
    f = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n, d=1.0 / n)
    s1 = 1j * (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h)
    s2 = -(30 - 32 * np.cos(k * h) + 2 * np.cos(2 * k * h)) / (12 * h * h)
    ft = torch.from_numpy(f)
    for axis, npax in ((0, 2), (1, 1), (2, 0)):
        shape = [1, 1, 1]
        shape[npax] = n
        g1 = np.real(np.fft.ifft(np.fft.fft(f, axis=npax) * s1.reshape(shape), axis=npax))
        g2 = np.real(np.fft.ifft(np.fft.fft(f, axis=npax) * s2.reshape(shape), axis=npax))
        assert np.allclose(oracle.d1(ft, axis, h).numpy(), g1, atol=1e-12)
        assert np.allclose(oracle.d2(ft, axis, h).numpy(), g2, atol=1e-10)


def test_mixed_derivative_is_product_of_symbols():
    n = 16
    h = 2 * math.pi / n
    c = torch.arange(n, dtype=torch.float64) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    kx, ky = 3, 5
    f = torch.exp(1j * (kx * x + ky * y).to(torch.complex128))
    s = lambda k: 1j * (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h)
    g = oracle.d1(oracle.d1(f, 1, h), 0, h)
    assert torch.allclose(g, s(kx) * s(ky) * f, atol=1e-11, rtol=0)


def test_fourth_order_convergence():
    errs1, errs2 = [], []
    for n in (16, 32, 64):
        x, y, z = oracle.grid(n)
        f = torch.sin(x + 2 * y) * torch.cos(z)
        h = 2 * math.pi / n
        errs1.append(float((oracle.d1(f, 0, h) - torch.cos(x + 2 * y) * torch.cos(z)).abs().max()))
        errs2.append(float((oracle.d2(f, 1, h) + 4 * f).abs().max()))
    for e in (errs1, errs2):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 14.0 < r2 < 17.0 and r1 > 12.0, e


def _read_rk_golden():
    rows = {}
    with open(os.path.join(GOLDEN, "rk3_williamson.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = [float(Fraction(v)) for v in vals]
    return rows


def test_rk_coefficients_are_the_golden_ones():
    g = _read_rk_golden()
    assert np.allclose(oracle.RK_A, g["A"], rtol=0, atol=1e-16)
    assert np.allclose(oracle.RK_B, g["B"], rtol=0, atol=1e-16)


def test_rk3_stability_polynomial():
    g = _read_rk_golden()["P"]
    flow = oracle.Flow(n=4)
    for lam_dt in (0.3, -1.0, 1.2j, -0.5 + 0.8j, -2.0 + 0.1j):
        lam = complex(lam_dt)
        q0 = torch.ones(5, 4, 4, 4, dtype=torch.complex128)
        q1 = oracle.rk3_step(flow, q0, 1.0, rhs=lambda q: lam * q)
        poly = sum(c * lam ** m for m, c in enumerate(g))
        assert abs(complex(q1[0, 0, 0, 0]) - poly) < 1e-14, lam_dt


def test_rk3_third_order_on_nonlinear_ode():
    # q' = -q^2, q(0) = 1  ->  q(t) = 1 / (1 + t)
    flow = oracle.Flow(n=4)
    errs = []
    for nsteps in (20, 40, 80):
        dt = 1.0 / nsteps
        q = torch.ones(5, 4, 4, 4, dtype=torch.float64)
        for _ in range(nsteps):
            q = oracle.rk3_step(flow, q, dt, rhs=lambda s: -s * s)
        errs.append(abs(float(q[0, 0, 0, 0]) - 0.5))
    assert 7.0 < errs[0] / errs[1] < 9.0 and 7.0 < errs[1] / errs[2] < 9.0, errs
