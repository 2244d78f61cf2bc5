"""GPU discrete adjoint against the FP64 oracle, the dot-product identity and
finite differences.

Gates (FP64): rhs_vjp equals the oracle's reverse-mode VJP to 1e-11 of each
component's scale; <J v, w> = <v, J^T w> to 1e-10 with J v from the oracle's
forward-mode JVP and J^T w from the GPU; the gradient of the final kinetic
energy equals the oracle's adjoint to 1e-10 and central differences of the
GPU forward map on 16 seeded directions (64^3, 200 steps, checkpoint every
20) to 1e-6.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import tgv_inputs
import paper_2505_20911_b300 as tgv
from _util import encode, oracle_flow, random_state

pytestmark = pytest.mark.gpu


def _rand(shape, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return torch.from_numpy(rng.standard_normal(shape))


@pytest.mark.parametrize("split,mu", [("blaisdell", 1.0), ("divergence", 1.0), ("blaisdell", 0.0)])
def test_rhs_vjp_matches_oracle(split, mu):
    cfg = tgv.Config(n=32, mode="fp64", mach=0.3, re=50.0, split=split, mu=mu)
    q64 = random_state(cfg, seed=31)
    lam = _rand(q64.shape, 32)
    got = torch.empty(q64.shape, dtype=torch.float64, device="cuda")
    tgv.rhs_vjp(cfg, encode(cfg, q64), lam.cuda(), got)
    ref = oracle.rhs_vjp(oracle_flow(cfg), q64, lam)
    for c in range(5):
        scale = float(ref[c].abs().max())
        assert float((got[c].cpu() - ref[c]).abs().max()) <= 1e-11 * scale, c


def test_rhs_dot_product_identity():
    """<J v, w> with J v from the oracle's forward mode, <v, J^T w> from the GPU."""
    cfg = tgv.Config(n=32, mode="fp64", mach=0.2, re=200.0)
    q64 = random_state(cfg, seed=41)
    v, w = _rand(q64.shape, 42), _rand(q64.shape, 43)
    jv = oracle.rhs_jvp(oracle_flow(cfg), q64, v)
    jtw = torch.empty(q64.shape, dtype=torch.float64, device="cuda")
    tgv.rhs_vjp(cfg, encode(cfg, q64), w.cuda(), jtw)
    a = float((jv * w).sum())
    b = float((v * jtw.cpu()).sum())
    assert abs(a - b) <= 1e-10 * abs(a), (a, b)


def _stage_inputs(cfg, q64, dt):
    """The three stage inputs of one GPU forward step from q64, stacked."""
    si = torch.empty((3,) + tuple(q64.shape), dtype=torch.float64, device="cuda")
    si[0] = q64.cuda()
    qt = tgv.empty_qt(cfg)
    tgv.rk_substep(cfg, si[0], si[1], qt, 0, dt)
    tgv.rk_substep(cfg, si[1], si[2], qt, 1, dt)
    return si


def test_rk_step_adjoint_matches_oracle_and_dot_product():
    cfg = tgv.Config(n=32, mode="fp64", mach=0.2, re=200.0)
    flow = oracle_flow(cfg)
    q64 = random_state(cfg, seed=51)
    dt = 0.004
    qbar_next = _rand(q64.shape, 52)
    qb = qbar_next.clone().cuda()
    tgv.rk_step_adjoint(cfg, _stage_inputs(cfg, q64, dt), qb, dt)
    # oracle: reverse mode through one RK3 step
    x = q64.clone().requires_grad_(True)
    out = oracle.rk3_step(flow, x, dt)
    (ref,) = torch.autograd.grad(out, x, grad_outputs=qbar_next)
    for c in range(5):
        assert float((qb[c].cpu() - ref[c]).abs().max()) <= 1e-10 * float(ref[c].abs().max()), c
    # dot product: <(dQ1/dQ0) v, w> from the oracle's forward mode
    v = _rand(q64.shape, 53)
    _, jv = torch.func.jvp(lambda s: oracle.rk3_step(flow, s, dt), (q64,), (v,))
    a = float((jv * qbar_next).sum())
    b = float((v * qb.cpu()).sum())
    assert abs(a - b) <= 1e-10 * abs(a), (a, b)


def _grad(cfg, q0, dt, nsteps, ckpt):
    g = torch.empty((3,) + tuple(q0.shape[1:]), dtype=torch.float64, device="cuda")
    j = torch.empty(1, dtype=torch.float64, device="cuda")
    tgv.tgv_grad_final_ke(cfg, q0, dt, nsteps, ckpt, g, j)
    torch.cuda.synchronize()
    return float(j[0]), g


def test_grad_final_ke_matches_oracle_adjoint():
    cfg = tgv.Config(n=32, mode="fp64", mach=0.2, re=400.0)
    flow = oracle_flow(cfg)
    q64 = oracle.initial_condition(flow)
    # break the Taylor-Green symmetries so every gradient component is exercised
    q64[1:4] += 0.05 * torch.from_numpy(np.stack(tgv_inputs.adjoint_directions(32, 1)[0]))
    dt, nsteps, ckpt = 0.004, 12, 5
    J, g = _grad(cfg, encode(cfg, q64), dt, nsteps, ckpt)
    J_ref, g_ref = oracle.grad_final_ke(flow, q64, dt, nsteps, ckpt_every=4)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    err = float(torch.linalg.vector_norm(g.cpu() - g_ref) / torch.linalg.vector_norm(g_ref))
    assert err <= 1e-10, err


def _broken_symmetry_ic(flow, n, seed_dirs=1):
    """The Taylor-Green field plus 0.05 of a seeded smooth momentum direction
    (so that no symmetry of the TGV hides a wrong gradient component)."""
    q = oracle.initial_condition(flow)
    q[1:4] += 0.05 * torch.from_numpy(np.stack(tgv_inputs.adjoint_directions(n, seed_dirs)[0]))
    return q


def test_grad_final_ke_matches_oracle_adjoint_64cubed():
    """The adjoint configuration's grid (64^3, FP64, dt = 0.004): 20 steps with a
    checkpoint every 5 against the oracle's reverse-mode adjoint."""
    cfg = tgv.Config(n=64, mode="fp64")
    flow = oracle_flow(cfg)
    q64 = _broken_symmetry_ic(flow, 64)
    dt, nsteps = 0.004, 20
    J, g = _grad(cfg, encode(cfg, q64), dt, nsteps, 5)
    J_ref, g_ref = oracle.grad_final_ke(flow, q64, dt, nsteps, ckpt_every=5)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    err = float(torch.linalg.vector_norm(g.cpu() - g_ref) / torch.linalg.vector_norm(g_ref))
    print(f"\n64^3 x 20 steps: |g - g_oracle| / |g_oracle| = {err:.2e}")
    assert err <= 1e-10, err


def _fp32_storage_step(flow, q, dt):
    """One RK3 step of the oracle's FP64 residual with the state and the
    increment stored in FP32 after every stage, as the FP32 mode's substeps
    store them: Qt <- A Qt + dt R, Q <- Q + B Qt (Sec. 3.1, Eqs. 3-4).  The
    rounding is a value-only correction, so reverse mode differentiates the
    FP64 map at the rounded states.  Returns the step's result and its three
    stage inputs (each exactly representable in FP32)."""
    r32 = lambda x: x + (x.detach().float().double() - x.detach())
    qt = torch.zeros_like(q)
    stages = []
    for i in range(3):
        stages.append(q)
        qt = r32(oracle.RK_A[i] * qt + dt * oracle.residual(flow, q))
        q = r32(q + oracle.RK_B[i] * qt)
    return q, stages


def test_fp32_forward_variant_adjoint_at_fp32_stage_states():
    """FP32 forward / FP64 adjoint: the step adjoint of the FP32 mode, given
    FP32 stage states, is the exact transpose of the FP64 step map linearised
    at those states.  The oracle makes an FP32-stored step of its own (64^3,
    symmetries broken) and differentiates it in reverse mode; the library's
    rk_step_adjoint gets the same three stage states in FP32 storage."""
    n, dt = 64, 0.004
    c32 = tgv.Config(n=n, mode="fp32")
    flow = oracle_flow(c32)
    q0 = _broken_symmetry_ic(flow, n).float().double()
    x = q0.clone().requires_grad_(True)
    out, stages = _fp32_storage_step(flow, x, dt)
    qbar_next = _rand(q0.shape, 61)
    (ref,) = torch.autograd.grad(out, x, grad_outputs=qbar_next)
    st64 = torch.stack([s_.detach() for s_ in stages])
    si = st64.float().cuda()
    assert torch.equal(si.double().cpu(), st64)     # the stage states are FP32 values
    qb = qbar_next.clone().cuda()
    tgv.rk_step_adjoint(c32, si, qb, dt)
    for c in range(5):
        err = float((qb[c].cpu() - ref[c]).abs().max()) / float(ref[c].abs().max())
        assert err <= 1e-10, (c, err)


def test_fp32_forward_variant_gradient_tracks_the_fp64_gradient():
    """The whole FP32-forward gradient (64^3, 10 steps, checkpoint every 5):
    its own FP32 trajectory differs from the FP64 one by FP32 rounding, so the
    gradient agrees with the oracle's FP64 adjoint to about 1e-6 (measured
    1.2e-6 against an FP32-stored oracle trajectory at this size), far inside
    the 1e-3 of the 200-step comparison."""
    n, dt, nsteps = 64, 0.004, 10
    c32 = tgv.Config(n=n, mode="fp32")
    flow = oracle_flow(c32)
    q0 = _broken_symmetry_ic(flow, n).float().double()
    J32, g32 = _grad(c32, encode(c32, q0), dt, nsteps, 5)
    J64, g64 = oracle.grad_final_ke(flow, q0, dt, nsteps, ckpt_every=5)
    err = float(torch.linalg.vector_norm(g32.cpu() - g64) / torch.linalg.vector_norm(g64))
    print(f"\nFP32 forward, 64^3 x 10 steps: |g32 - g64_oracle| / |g64_oracle| = {err:.2e}")
    assert abs(J32 - J64) <= 1e-6 * abs(J64)
    assert err <= 1e-5, err


def _final_ke_gpu(cfg, q0, dt, nsteps):
    qa = q0.clone()
    qb = torch.empty_like(qa)
    qt = tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, dt, nsteps)
    return tgv.diagnostics(cfg, qb if par else qa)["K"]


def test_grad_final_ke_fd_16_directions_64cubed():
    """The adjoint configuration: 64^3 TGV, FP64, 200 RK3 steps at dt = 0.004,
    checkpoint every 20 steps; central differences on 16 seeded directions."""
    cfg = tgv.Config(n=64, mode="fp64")
    q0 = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q0)
    dt, nsteps, ckpt = 0.004, 200, 20
    J, g = _grad(cfg, q0, dt, nsteps, ckpt)
    assert abs(J - _final_ke_gpu(cfg, q0, dt, nsteps)) <= 1e-14 * J
    rms = float(torch.sqrt((q0[1:4] ** 2).mean()))
    # J is O(0.1) and these directional derivatives are O(1e-6): the FP64
    # rounding noise of J (about 1e-16 absolute) limits small steps, so take a
    # larger step with a 4th-order difference (truncation O(eps^4))
    eps = 1e-3 * rms
    worst = 0.0
    gnorm = float(torch.linalg.vector_norm(g))
    for d in tgv_inputs.adjoint_directions(64, 16):
        v = torch.zeros_like(q0)
        v[1:4] = torch.from_numpy(d).cuda()
        J_ = {m: _final_ke_gpu(cfg, q0 + m * eps * v, dt, nsteps) for m in (-2, -1, 1, 2)}
        fd = (8.0 * (J_[1] - J_[-1]) - (J_[2] - J_[-2])) / (12.0 * eps)
        ad = float((g * v[1:4]).sum())
        # error scale: |ad| itself, or (for directions nearly orthogonal to the
        # gradient, where ad ~ 1e-10) the largest directional derivative |g||v|
        scale = max(abs(ad), 1e-2 * gnorm * float(torch.linalg.vector_norm(v)))
        worst = max(worst, abs(fd - ad) / scale)
        assert abs(fd - ad) <= 1e-6 * scale, (fd, ad, scale)
    print(f"worst FD mismatch over 16 directions: {worst:.2e} of max(|ad|, 0.01 |g||v|)")


def test_fp32_forward_fp64_adjoint_variant():
    """FP32 forward states with the FP64 adjoint: the gradient stays close to
    the FP64 one (the difference is the FP32 trajectory error, O(1e-5) here)."""
    n, dt, nsteps, ckpt = 64, 0.004, 200, 20
    c64 = tgv.Config(n=n, mode="fp64")
    c32 = tgv.Config(n=n, mode="fp32")
    q64 = tgv.empty_state(c64)
    tgv.tgv_init(c64, q64)
    q32 = tgv.empty_state(c32)
    tgv.tgv_init(c32, q32)
    J64, g64 = _grad(c64, q64, dt, nsteps, ckpt)
    J32, g32 = _grad(c32, q32, dt, nsteps, ckpt)
    assert abs(J32 - J64) <= 1e-5 * J64
    err = float(torch.linalg.vector_norm(g32 - g64) / torch.linalg.vector_norm(g64))
    assert err <= 1e-3, err


def test_autograd_function_backward():
    cfg = tgv.Config(n=32, mode="fp64")
    q0 = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q0)
    ru, rv, rw = (q0[c].clone().requires_grad_(True) for c in (1, 2, 3))
    J = tgv.TGVFinalKE.apply(ru, rv, rw, q0[0], q0[4], cfg, 0.004, 10, 5)
    J.backward()
    _, g = _grad(cfg, q0, 0.004, 10, 5)
    for a, b in ((ru.grad, g[0]), (rv.grad, g[1]), (rw.grad, g[2])):
        assert torch.equal(a, b)
