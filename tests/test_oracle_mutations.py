"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in the oracle (a wrong sign, a dropped term, a
transposed axis, a wrong coefficient) with monkeypatch and checks that the
pin meant to guard that part now fails.
"""
import math

import pytest
import torch

import oracle
import oracle.tgv_oracle as T
from test_oracle_rhs import _errors, _exact_groups, _random_state


@pytest.fixture(scope="module")
def exact():
    return _exact_groups()


def _converges(exact, group):
    e32, e64 = _errors(exact, group, 32), _errors(exact, group, 64)
    for c in range(5):
        (a, scale), (b, _) = e32[c], e64[c]
        if scale < 1e-12:
            if a > 1e-12 or b > 1e-12:
                return False
            continue
        if not (b < 1e-3 * scale and a / b > 13.0):
            return False
    return True


def test_unmutated_oracle_passes(exact):
    assert _converges(exact, "total")


def test_wrong_sign_of_pressure_work_is_caught(exact, monkeypatch):
    orig = T.pressure_terms

    def bad(flow, q):
        r = orig(flow, q).clone()
        r[4] = -r[4]
        return r
    monkeypatch.setattr(T, "pressure_terms", bad)
    monkeypatch.setattr(oracle, "pressure_terms", bad)
    assert not _converges(exact, "total")


def test_transposed_axis_is_caught(exact, monkeypatch):
    orig = T.d1
    monkeypatch.setattr(T, "d1", lambda f, axis, h: orig(f, {0: 0, 1: 2, 2: 1}[axis], h))
    assert not _converges(exact, "convective")


def test_dropped_dilatation_cross_term_is_caught(exact, monkeypatch):
    orig = T.viscous_terms

    def bad(flow, q):
        r = orig(flow, q).clone()
        _, u, v, w, _, _ = T.primitives(flow, q)
        vel, h = (u, v, w), flow.h
        diag = [T.d1(vel[k], k, h) for k in range(3)]
        for i in range(3):
            s = sum(diag[k] for k in range(3) if k != i)
            r[1 + i] -= flow.mu / flow.re * T.d1(s, i, h) / 3.0
        return r
    monkeypatch.setattr(T, "viscous_terms", bad)
    monkeypatch.setattr(oracle, "viscous_terms", bad)
    assert not _converges(exact, "viscous")


def test_wrong_heat_conductivity_is_caught(exact, monkeypatch):
    monkeypatch.setattr(T.Flow, "kappa", property(
        lambda self: self.mu / ((self.gamma - 1.0) * self.mach ** 2 * self.re)))
    assert not _converges(exact, "viscous")


def test_dropped_blaisdell_term_is_caught(monkeypatch):
    orig = T.convective

    def bad(flow, q):
        r = orig(flow, q).clone()
        rho = q[0]
        div = sum(T.d1(q[1 + j] / rho, j, flow.h) for j in range(3))
        return r - 0.5 * q * div
    flow, q = _random_state(16, 5)
    rho = q[0]
    div = sum(oracle.d1(q[1 + j] / rho, j, flow.h) for j in range(3))
    conv = bad(flow, q)
    c = 2
    lhs = float((q[c] * conv[c]).sum())
    rhs = float((0.5 * div * q[c] * q[c]).sum())
    assert abs(lhs - rhs) > 1e-6 * float((q[c] * q[c]).sum())


def test_wrong_second_derivative_coefficient_is_caught():
    n, h, k = 16, 2 * math.pi / 16, 3
    c = torch.arange(n, dtype=torch.float64) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    f = torch.exp(1j * k * x.to(torch.complex128))
    bad = lambda g: (-T.shift(g, 0, 2) + 16 * T.shift(g, 0, 1) - 31 * g
                     + 16 * T.shift(g, 0, -1) - T.shift(g, 0, -2)) / (12 * h * h)
    sym = -(30 - 32 * math.cos(k * h) + 2 * math.cos(2 * k * h)) / (12 * h * h)
    assert not torch.allclose(bad(f), sym * f, atol=1e-11, rtol=0)


def test_wrong_rk_coefficient_is_caught(monkeypatch):
    monkeypatch.setattr(T, "RK_B", (1.0 / 3.0, 15.0 / 16.0, 8.0 / 16.0))
    flow = oracle.Flow(n=4)
    lam = -0.5 + 0.8j
    q0 = torch.ones(5, 4, 4, 4, dtype=torch.complex128)
    q1 = T.rk3_step(flow, q0, 1.0, rhs=lambda q: lam * q)
    poly = 1 + lam + lam ** 2 / 2 + lam ** 3 / 6
    assert abs(complex(q1[0, 0, 0, 0]) - poly) > 1e-3
