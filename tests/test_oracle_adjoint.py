"""Pins of the oracle's discrete adjoint and of its inviscid behaviour (CPU).

The adjoint (gradient of the final volume-averaged kinetic energy, Sec. 4.1
Eq. 11, with respect to the initial momentum) is pinned by central finite
differences of the oracle's own forward map and by the dot-product identity
<J v, w> = <v, J^T w> between forward- and reverse-mode derivatives.
"""
import numpy as np
import torch

import oracle
import tgv_inputs


def _flow_and_q0(n=16, mach=0.1, re=1600.0):
    flow = oracle.Flow(n=n, mach=mach, re=re)
    return flow, oracle.initial_condition(flow)


def test_gradient_matches_central_differences():
    flow, q0 = _flow_and_q0(16, mach=0.2, re=400.0)
    dt, nsteps = 0.004, 6
    J, g = oracle.grad_final_ke(flow, q0, dt, nsteps, ckpt_every=3)
    assert abs(J - float(oracle.final_ke(flow, q0, dt, nsteps))) < 1e-15
    for d in tgv_inputs.adjoint_directions(16, count=3):
        v = torch.zeros_like(q0)
        v[1:4] = torch.from_numpy(d)
        eps = 1e-5
        jp = float(oracle.final_ke(flow, q0 + eps * v, dt, nsteps))
        jm = float(oracle.final_ke(flow, q0 - eps * v, dt, nsteps))
        fd = (jp - jm) / (2 * eps)
        ad = float((g * v[1:4]).sum())
        assert abs(fd - ad) < 1e-7 * abs(ad) + 1e-12, (fd, ad)


def test_checkpoint_interval_does_not_change_gradient():
    flow, q0 = _flow_and_q0(16)
    _, g1 = oracle.grad_final_ke(flow, q0, 0.004, 5, ckpt_every=1)
    _, g5 = oracle.grad_final_ke(flow, q0, 0.004, 5, ckpt_every=5)
    assert torch.equal(g1, g5)


def test_rhs_dot_product_identity():
    flow = oracle.Flow(n=16, mach=0.3, re=50.0)
    rho, u, v, w, dp = (torch.from_numpy(a) for a in tgv_inputs.random_flow_fields(16, 11))
    q = oracle.conserved(flow, rho, u, v, w, 1.0 / (1.4 * 0.09) + dp)
    rng = np.random.Generator(np.random.PCG64(5))
    vv = torch.from_numpy(rng.standard_normal(q.shape))
    ww = torch.from_numpy(rng.standard_normal(q.shape))
    jv = oracle.rhs_jvp(flow, q, vv)
    jtw = oracle.rhs_vjp(flow, q, ww)
    a, b = float((jv * ww).sum()), float((vv * jtw).sum())
    assert abs(a - b) < 1e-12 * abs(a), (a, b)


def test_inviscid_kinetic_energy_is_nearly_conserved():
    # Inviscid TGV, M = 0.4, dt = 0.004 (the setting of Sec. 4.2's split-form
    # study, on a coarser grid): the Blaisdell split keeps K/K0 close to 1.
    flow = oracle.Flow(n=32, mach=0.4, mu=0.0)
    q = oracle.initial_condition(flow)
    k0 = float(oracle.kinetic_energy(flow, q))
    worst = 0.0
    for _ in range(250):
        q = oracle.rk3_step(flow, q, 0.004)
        worst = max(worst, abs(float(oracle.kinetic_energy(flow, q)) / k0 - 1.0))
    assert worst < 2e-3, worst
