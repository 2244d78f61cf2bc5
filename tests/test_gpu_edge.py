"""Edge cases of the CUDA path: the smallest and the largest grids the library
accepts, grids smaller than one CTA tile, no steps, a zero time step, and the
uniform states whose residual vanishes exactly."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2505_20911_b300 as tgv
from _util import decode, encode, max_rel, oracle_flow, random_state, window, window_flow

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [8, 10])
def test_grids_smaller_than_one_tile(mode, n):
    """N = 8 (the minimum) and 10: one CTA covers the whole plane and the
    periodic halo wraps inside the tile; residual and 3 steps against the oracle."""
    cfg = tgv.Config(n=n, mode=mode, mach=0.3, re=50.0)
    flow = oracle_flow(cfg)
    q64 = random_state(cfg, seed=100 + n)
    r = torch.empty(5, n, n, n, dtype=cfg.q_dtype, device="cuda")
    tgv.rhs_eval(cfg, encode(cfg, q64), r)
    tol = 1e-11 if mode == "fp64" else 2e-4
    assert max(max_rel(r.double().cpu(), oracle.residual(flow, q64))) < tol
    qa = encode(cfg, q64)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, 0.002, 3)
    ref = oracle.run(flow, q64, 0.002, 3)
    got = decode(cfg, qb if par else qa)
    assert max(max_rel(got, ref)) < (1e-13 if mode == "fp64" else 1e-5)


def test_symmetric_box_smaller_than_one_tile():
    cfg = tgv.Config(n=8, mode="fp32", length=math.pi, symmetric=True, mach=0.5, re=800.0)
    flow = oracle_flow(cfg)
    q64 = oracle.initial_condition(flow)
    r = torch.empty(5, 8, 8, 8, dtype=torch.float32, device="cuda")
    tgv.rhs_eval(cfg, encode(cfg, q64), r)
    ref = oracle.residual(flow, q64)
    assert max(max_rel(r.double().cpu(), ref)) < 2e-4


@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp16_fp32"])
def test_zero_steps_leave_the_state_alone(mode):
    cfg = tgv.Config(n=16, mode=mode)
    qa = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, qa)
    qb = torch.full_like(qa, 7.0)
    keep_a, keep_b = qa.clone(), qb.clone()
    par = tgv.rk_step(cfg, qa, qb, tgv.empty_qt(cfg), 0.004, 0)
    assert par == 0
    assert torch.equal(qa, keep_a) and torch.equal(qb, keep_b)


@pytest.mark.parametrize("mode", ["fp64", "spdp", "fp32", "hpsp", "bf16_fp32", "fp16_fp32", "fp16"])
def test_zero_time_step_is_the_identity(mode):
    """dt = 0: every increment is a signed zero, so the three substeps return
    the input state value for value, offset encoding included."""
    cfg = tgv.Config(n=24, mode=mode, encoding="offset" if mode in ("bf16_fp32", "fp16_fp32", "fp16")
                     else "plain")
    qa = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, qa)
    keep = qa.clone()
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    bufs = [qa, qb]
    for i in range(3):
        tgv.rk_substep(cfg, bufs[i % 2], bufs[(i + 1) % 2], qt, i, 0.0)
    assert torch.equal(qb, keep)
    assert float(qt.abs().max()) == 0.0


@pytest.mark.parametrize("mode", ["fp64", "spdp", "fp32", "hpsp", "bf16_fp32", "fp16_fp32", "fp16"])
@pytest.mark.parametrize("velocity", [(0.0, 0.0, 0.0), (0.25, -0.125, 0.5)])
def test_uniform_state_has_a_zero_residual(mode, velocity):
    """A uniform state (at rest or in uniform translation) is a steady solution,
    and every stencil applied to equal taps cancels exactly in floating point:
    R is exactly zero and steps leave the state unchanged."""
    n = 24
    cfg = tgv.Config(n=n, mode=mode, mach=0.2)
    flow = oracle_flow(cfg)
    one = torch.ones(n, n, n, dtype=torch.float64)
    p0 = 1.0 / (cfg.gamma * cfg.mach ** 2)
    q64 = oracle.conserved(flow, one, velocity[0] * one, velocity[1] * one, velocity[2] * one, p0 * one)
    q = encode(cfg, q64)
    if mode in ("fp64", "fp32"):
        r = torch.empty(5, n, n, n, dtype=cfg.q_dtype, device="cuda")
        tgv.rhs_eval(cfg, q, r)
        assert float(r.abs().max()) == 0.0
    keep = q.clone()
    qb, qt = torch.empty_like(q), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, q, qb, qt, 0.004, 4)
    assert torch.equal(qb if par else q, keep)
    if mode in ("fp64", "fp32", "fp16_fp32"):
        sym = cfg.with_(length=math.pi, symmetric=True)
        if velocity == (0.0, 0.0, 0.0):
            q = keep.clone()
            par = tgv.rk_step(sym, q, qb, qt, 0.004, 4)
            assert torch.equal(qb if par else q, keep)


def test_largest_grid_half_single_stage_sampled():
    """N = 1024, the largest grid the library accepts (5 fields x 2^30 points,
    so every field offset above 2^31 elements), in the benchmark's half-single
    mode: Qt after the first substep at sampled points against the oracle on a
    periodic window around each point.  Same bound as the 256^3/512^3 test."""
    cfg = tgv.Config(n=1024, mode="fp16_fp32", encoding="offset")
    dt = 0.0003
    qa = tgv.empty_state(cfg)
    qb = torch.empty_like(qa)
    qt = tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    tgv.rk_substep(cfg, qa, qb, qt, 0, dt)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(1024))
    wf = window_flow(cfg)
    got, ref = [], []
    pts = [(int(a), int(b), int(c)) for a, b, c in rng.integers(0, cfg.n, size=(20, 3))]
    pts += [(0, 0, 0), (1023, 1023, 1023), (1023, 0, 511)]
    for k, j, i in pts:
        w = decode(cfg, window(qa, k, j, i))
        ref.append(dt * oracle.residual(wf, w)[:, 4, 4, 4])
        got.append(qt[:, k, j, i].double().cpu())
    got, ref = torch.stack(got), torch.stack(ref)
    h = cfg.length / cfg.n
    big = 1.0 / (cfg.gamma * (cfg.gamma - 1) * cfg.mach ** 2) + 1.0 / (cfg.gamma * cfg.mach ** 2)
    mag = torch.tensor([4.0, big + 4, big + 4, big + 4, big + 4], dtype=torch.float64)
    bound = 4 * dt * 2.0 ** -24 * mag * 1.5 / h
    assert bool(((got - ref).abs() <= 2.0 ** -10 * ref.abs() + bound).all())
    # the far corner of the last field was written (offsets past 2^32 bytes)
    assert bool(torch.isfinite(qb[4, -1, -1, -8:].float()).all())
