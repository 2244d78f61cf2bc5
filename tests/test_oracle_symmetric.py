"""Pins of the oracle's symmetric box (the TGSym domain of Sec. 4.1; reading
R13: [0, L]^3 with a mirror plane on every face, cell-centred points)."""
import math

import torch

import oracle


def _flows(n, **kw):
    sym = oracle.Flow(n=n, length=math.pi, symmetric=True, **kw)
    twin = oracle.Flow(n=2 * n, length=2 * math.pi, offset=0.5, **kw)
    return sym, twin


def test_initial_field_is_one_octant_of_the_periodic_one():
    sym, twin = _flows(16, mach=0.5, re=800.0)
    q = oracle.initial_condition(sym)
    assert torch.allclose(oracle.mirror_extend(q), oracle.initial_condition(twin), atol=1e-14, rtol=0)


def test_periodic_twin_keeps_the_mirror_structure():
    """The periodic scheme maps mirror-symmetric states to mirror-symmetric
    states (the discrete operator commutes with the reflections), so the
    symmetric box's solution is the restriction of the periodic one."""
    sym, twin = _flows(12, mach=0.5, re=200.0)
    q = oracle.initial_condition(twin)
    for _ in range(5):
        q = oracle.rk3_step(twin, q, 0.004)
    n = 12
    ext = oracle.mirror_extend(q[:, :n, :n, :n])
    assert torch.allclose(ext, q, rtol=0, atol=1e-12 * float(q.abs().max()))
    # and the symmetric oracle reproduces the restriction step by step
    qs = oracle.initial_condition(sym)
    for _ in range(5):
        qs = oracle.rk3_step(sym, qs, 0.004)
    assert torch.allclose(qs, q[:, :n, :n, :n], rtol=0, atol=1e-12 * float(q.abs().max()))


def test_symmetric_box_closed_forms_and_conservation():
    sym, _ = _flows(16, mach=0.5, re=800.0)
    q = oracle.initial_condition(sym)
    d0 = oracle.diagnostics(sym, q)
    # cell-centred sampling of sin^2 and cos^2 over [0, pi] averages to 1/2 exactly
    assert abs(d0["K"] - 0.125) < 1e-15 and abs(d0["rho"] - 1.0) < 1e-15
    for _ in range(5):
        q = oracle.rk3_step(sym, q, 0.004)
    d1 = oracle.diagnostics(sym, q)
    # mirror planes are impermeable and adiabatic: mass and total energy stay put
    assert abs(d1["rho"] - d0["rho"]) < 1e-14
    assert abs(d1["rho_E"] - d0["rho_E"]) < 1e-13 * d0["rho_E"]
