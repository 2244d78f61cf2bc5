"""Pins of the oracle's initial condition, diagnostics and short-time behaviour.

Closed forms come from tests/golden/tgv_closed_forms.txt (derived from
Sec. 4.1, Eqs. 6-12).
"""
import math
import os

import pytest
import torch

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    vals = {}
    with open(os.path.join(GOLDEN, "tgv_closed_forms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, n, val = line.split()
            vals[(key, n)] = float(val)
    return vals


@pytest.mark.parametrize("n", [16, 32, 48])
@pytest.mark.parametrize("mach", [0.1, 0.5])
def test_initial_condition_closed_forms(n, mach):
    g = _golden()
    flow = oracle.Flow(n=n, mach=mach)
    q = oracle.initial_condition(flow)
    rho, u, v, w, p, T = oracle.primitives(flow, q)
    d = oracle.diagnostics(flow, q)
    assert abs(d["K"] - g[("K0", "any")]) < 1e-15
    assert abs(d["K_rho"] - g[("K_rho0", "any")]) < 1e-15
    assert abs(d["rho"] - g[("rho_mean", "any")]) < 1e-15
    assert float((T - g[("T0", "any")]).abs().max()) < 1e-13
    assert float(w.abs().max()) == 0.0
    if ("enstrophy0", str(n)) in g:
        assert abs(d["enstrophy"] - g[("enstrophy0", str(n))]) < 1e-13
        assert abs(d["eps_S"] - g[("enstrophy0", str(n))] / flow.re) < 1e-16
    assert d["nonfinite"] == 0.0


def test_initial_field_pointwise():
    flow = oracle.Flow(n=16, mach=0.1)
    q = oracle.initial_condition(flow)
    x, y, z = oracle.grid(16)
    rho, u, v, w, p, T = oracle.primitives(flow, q)
    assert torch.allclose(u, torch.sin(x) * torch.cos(y) * torch.cos(z), atol=1e-14)
    assert torch.allclose(v, -torch.cos(x) * torch.sin(y) * torch.cos(z), atol=1e-14)
    pref = 1 / (1.4 * 0.01) + (torch.cos(2 * x) + torch.cos(2 * y)) * (2 + torch.cos(2 * z)) / 16
    assert torch.allclose(p, pref, rtol=1e-14, atol=0)
    assert torch.allclose(rho, 1.4 * 0.01 * pref, rtol=1e-14, atol=0)


def test_discrete_continuity_of_initial_field():
    flow = oracle.Flow(n=32)
    _, u, v, w, _, _ = oracle.primitives(flow, oracle.initial_condition(flow))
    div = oracle.d1(u, 0, flow.h) + oracle.d1(v, 1, flow.h) + oracle.d1(w, 2, flow.h)
    assert float(div.abs().max()) < 1e-13


def test_initial_decay_rate_matches_dissipation():
    # Near-incompressible limit: dK/dt(0) = -<omega.omega>/Re up to O(M^2) and
    # the viscous stress of the dilatation (Sec. 4.1, text after Eq. 12).
    flow = oracle.Flow(n=32, mach=0.1, re=100.0)
    q0 = oracle.initial_condition(flow)
    dt = 1e-4
    k = [oracle.kinetic_energy(flow, q0)]
    q = q0
    for _ in range(2):
        q = oracle.rk3_step(flow, q, dt)
        k.append(oracle.kinetic_energy(flow, q))
    dkdt = float(-3 * k[0] + 4 * k[1] - k[2]) / (2 * dt)   # one-sided 2nd order
    eps0 = oracle.diagnostics(flow, q0)["eps_S"]
    assert abs(dkdt + eps0) < 0.01 * eps0, (dkdt, eps0)


def test_conservation_over_steps():
    flow = oracle.Flow(n=16, mach=0.1, re=1600.0)
    q = oracle.initial_condition(flow)
    d0 = oracle.diagnostics(flow, q)
    for _ in range(20):
        q = oracle.rk3_step(flow, q, 0.004)
    d1 = oracle.diagnostics(flow, q)
    assert abs(d1["rho"] - d0["rho"]) < 1e-14
    for k in ("rho_u", "rho_v", "rho_w"):
        assert abs(d1[k] - d0[k]) < 1e-14
    assert abs(d1["rho_E"] - d0["rho_E"]) < 1e-13 * d0["rho_E"]


def test_symmetries_persist_over_steps():
    from test_oracle_rhs import _tgv_symmetry_ops
    flow = oracle.Flow(n=16, mach=0.1, re=1600.0)
    q = oracle.initial_condition(flow)
    for _ in range(10):
        q = oracle.rk3_step(flow, q, 0.004)
    for op in _tgv_symmetry_ops(16):
        assert torch.allclose(op(q), q, rtol=0, atol=1e-12 * float(q.abs().max()))


def test_nonfinite_count_counts_points_not_components():
    """The oracle's non-finite diagnostic is the number of grid points where
    any of the 5 components is NaN or +-Inf: plant 4 bad values at 3 points
    (two components at one point) and 1 huge finite value."""
    flow = oracle.Flow(n=8)
    q = oracle.initial_condition(flow)
    q[0, 1, 2, 3] = float("nan")
    q[4, 1, 2, 3] = float("inf")          # same point as the NaN
    q[2, 5, 0, 7] = float("-inf")
    q[3, 7, 7, 0] = float("nan")
    q[1, 0, 0, 0] = 1e300                 # finite
    assert oracle.diagnostics(flow, q)["nonfinite"] == 3.0
