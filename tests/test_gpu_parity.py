"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 gates: the residual to 1e-11 of each field's scale, the initial field to
1e-14, and the state after 100 RK3 steps at 32^3 to 1e-10 relative field L2.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2505_20911_b300 as tgv
from _util import decode, encode, max_rel, oracle_flow, random_state, rel_l2, window, window_flow

pytestmark = pytest.mark.gpu


def test_initial_condition_matches_oracle():
    for n in (32, 40):
        cfg = tgv.Config(n=n, mode="fp64")
        q = tgv.empty_state(cfg)
        tgv.tgv_init(cfg, q)
        ref = oracle.initial_condition(oracle_flow(cfg))
        err = max_rel(decode(cfg, q), ref)
        assert max(err[:3] + err[4:]) < 1e-14, err
        assert float(q[3].abs().max()) == 0.0


@pytest.mark.parametrize("tile", [1, 2, 3])
@pytest.mark.parametrize("n,field", [(32, "tgv"), (32, "random"), (40, "random"), (48, "random")])
def test_rhs_fp64_matches_oracle(tile, n, field):
    cfg = tgv.Config(n=n, mode="fp64", tile=tile, mach=0.3 if field == "random" else 0.1,
                     re=50.0 if field == "random" else 1600.0)
    flow = oracle_flow(cfg)
    q64 = oracle.initial_condition(flow) if field == "tgv" else random_state(cfg, seed=n + tile)
    q = encode(cfg, q64)
    r = torch.empty_like(q)
    tgv.rhs_eval(cfg, q, r)
    torch.cuda.synchronize()
    ref = oracle.residual(flow, q64)
    err = max_rel(r.cpu(), ref)
    assert max(err) < 1e-11, err


@pytest.mark.parametrize("split", ["blaisdell", "divergence", "feiereisen", "kgp", "keep"])
@pytest.mark.parametrize("zchunk", [0, 5, 16])
def test_rhs_split_forms_and_zchunks(split, zchunk):
    cfg = tgv.Config(n=32, mode="fp64", split=split, zchunk=zchunk, mach=0.3, re=50.0)
    q64 = random_state(cfg, seed=7)
    r = torch.empty(5, 32, 32, 32, dtype=torch.float64, device="cuda")
    tgv.rhs_eval(cfg, encode(cfg, q64), r)
    ref = oracle.residual(oracle_flow(cfg), q64)
    assert max(max_rel(r.cpu(), ref)) < 1e-11


def test_inviscid_rhs():
    cfg = tgv.Config(n=32, mode="fp64", mu=0.0, mach=0.4)
    q64 = random_state(cfg, seed=3)
    r = torch.empty(5, 32, 32, 32, dtype=torch.float64, device="cuda")
    tgv.rhs_eval(cfg, encode(cfg, q64), r)
    ref = oracle.residual(oracle_flow(cfg), q64)
    assert max(max_rel(r.cpu(), ref)) < 1e-11


def test_substeps_match_oracle():
    cfg = tgv.Config(n=32, mode="fp64", mach=0.3, re=50.0)
    flow = oracle_flow(cfg)
    q64 = random_state(cfg, seed=11)
    qa, qb = encode(cfg, q64), torch.empty(5, 32, 32, 32, dtype=torch.float64, device="cuda")
    qt = tgv.empty_qt(cfg)
    dt = 0.002
    qo, qto = q64, torch.zeros_like(q64)
    bufs = [qa, qb]
    for i in range(3):
        tgv.rk_substep(cfg, bufs[i % 2], bufs[(i + 1) % 2], qt, i, dt)
        qo, qto = oracle.rk_substep(flow, qo, qto, i, dt)
        torch.cuda.synchronize()
        assert max(rel_l2(bufs[(i + 1) % 2].cpu(), qo)) < 1e-13
        assert max(rel_l2(qt.cpu(), qto)) < 1e-11


def test_fp64_100_steps_within_1e10():
    """The FP64 gate: 32^3 TGV, M=0.1, Re=1600, Pr=0.71, dt=0.004, 100 steps."""
    cfg = tgv.Config(n=32, mode="fp64")
    flow = oracle_flow(cfg)
    qa = tgv.empty_state(cfg)
    qb = torch.empty_like(qa)
    qt = tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    ws = tgv.empty_workspace(cfg)
    diag = torch.empty(11, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    par = tgv.rk_step(cfg, qa, qb, qt, 0.004, 100, diag_every=10, diag=diag, workspace=ws)
    assert par == 0
    q_ref, log = oracle.run(flow, oracle.initial_condition(flow), 0.004, 100, log_every=10)
    err = rel_l2(qa.cpu(), q_ref)
    assert max(err) < 1e-10, err
    d = diag.cpu().numpy()
    for rec, (step, ref) in enumerate(log):
        for m, name in enumerate(tgv.DIAG_NAMES):
            tol = 1e-12 * max(abs(ref[name]), 1e-300) + 1e-15
            assert abs(d[rec, m] - ref[name]) <= tol, (step, name, d[rec, m], ref[name])


def test_diagnostics_match_oracle_on_random_state():
    cfg = tgv.Config(n=40, mode="fp64", mach=0.3, re=50.0)
    q64 = random_state(cfg, seed=5)
    q64[1, 3, 4, 5] = float("nan")
    q64[4, 7, 7, 7] = float("inf")
    q64[0, 7, 7, 7] = float("-inf")       # a second bad component at the same point
    got = tgv.diagnostics(cfg, encode(cfg, q64))
    assert got["nonfinite"] == oracle.diagnostics(oracle_flow(cfg), q64)["nonfinite"] == 2.0
    q64[0, 7, 7, 7] = 1.0
    q64[1, 3, 4, 5] = 0.1
    q64[4, 7, 7, 7] = 50.0
    got = tgv.diagnostics(cfg, encode(cfg, q64))
    ref = oracle.diagnostics(oracle_flow(cfg), q64)
    for name in tgv.DIAG_NAMES:
        assert abs(got[name] - ref[name]) <= 1e-12 * abs(ref[name]) + 1e-15, name


def _sampled_first_substep(cfg, dt, samples=24):
    qa = tgv.empty_state(cfg)
    qb = torch.empty_like(qa)
    qt = tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    tgv.rk_substep(cfg, qa, qb, qt, 0, dt)
    torch.cuda.synchronize()
    q_in = decode(cfg, qa)
    rng = np.random.Generator(np.random.PCG64(cfg.n))
    wf = window_flow(cfg)
    got, ref = [], []
    for _ in range(samples):
        k, j, i = (int(v) for v in rng.integers(0, cfg.n, size=3))
        r = oracle.residual(wf, window(q_in, k, j, i))[:, 4, 4, 4]
        ref.append(dt * r)
        got.append(qt[:, k, j, i].double().cpu())
    del qa, qb, qt
    torch.cuda.empty_cache()
    return torch.stack(got), torch.stack(ref)


def test_full_size_fp64_stage_sampled():
    """256^3 in FP64: Qt after the first substep equals dt R(Q) at sampled
    points (oracle on a periodic window around each point)."""
    got, ref = _sampled_first_substep(tgv.Config(n=256, mode="fp64"), 0.00125)
    scale = ref.abs().max(dim=0).values
    assert bool(((got - ref).abs() <= 1e-11 * scale).all())


@pytest.mark.parametrize("n", [256, 512])
def test_full_size_half_single_stage_sampled(n):
    """Full-size grids in the benchmark's launch configuration (half-single,
    offset encoding): Qt after the first substep at sampled points.

    Bound from the arithmetic: FP32 rounding (u = 2^-24) of stencil taps whose
    magnitude is up to rho E + p (about 250 at M = 0.1) for the momentum and
    energy components (pressure and energy fluxes), or about 4 (rho u_j phi
    products) for mass, amplified by the first-derivative weights sum(|c|)/12h
    = 1.5/h, four such sums at most, times dt; plus the FP16 rounding of Qt
    (2^-11 relative)."""
    cfg = tgv.Config(n=n, mode="fp16_fp32", encoding="offset")
    dt = 0.000625
    got, ref = _sampled_first_substep(cfg, dt)
    h = cfg.length / n
    big = 1.0 / (cfg.gamma * (cfg.gamma - 1) * cfg.mach ** 2) + 1.0 / (cfg.gamma * cfg.mach ** 2)
    mag = torch.tensor([4.0, big + 4, big + 4, big + 4, big + 4], dtype=torch.float64)
    bound = 4 * dt * 2.0 ** -24 * mag * 1.5 / h
    assert bool(((got - ref).abs() <= 2.0 ** -10 * ref.abs() + bound).all())


def _rk3_step_stored(flow, q, dt, enc, dec):
    """One oracle RK3 step whose stage outputs and increments are rounded to a
    storage type where rk_step stores them: Q after each stage (through enc /
    dec) and the increment, kept divided by dt, after stages 1 and 2 (FP16
    here).  The arithmetic is the oracle's FP64."""
    w = torch.zeros_like(q)
    for s in range(3):
        w = oracle.RK_A[s] * w + oracle.residual(flow, q)
        if s < 2:
            w = w.half().double()
        q = dec(enc(q + oracle.RK_B[s] * dt * w))
    return q


@pytest.mark.parametrize("mode", ["fp16_fp32", "fp32"])
def test_full_size_rk_step_sampled(mode):
    """The benchmark's launch configuration end to end: one full rk_step at
    256^3 (the headline half-single mode with offset encoding, and FP32), at
    sampled points, against the oracle on a 16^3 periodic window around each
    point (three stages of radius-2 stencils reach 6 points: the window's
    centre is exact).
    FP32: against the plain oracle step; bound: three FP32 roundings of the
    stored value plus FP32 arithmetic on the pressure-dominated fluxes (as in
    the first-substep test).
    FP16 storage: the roundings of the stored stage states are not small next
    to the increments (the energy's f div u term multiplies the momentum's
    rounding by rho E ~ 180), so the reference is the oracle step with its
    stage states and increments rounded to FP16 where rk_step stores them.
    Most stored values then agree exactly; FP32 against FP64 arithmetic may
    flip the rounding of an intermediate store at a neighbour, one ulp of its
    momentum (2^-11 of it), which the energy's rho E div u term (weight
    rho E / 2 * 8 / (12 h) on the nearest neighbour) and the stage weight
    B dt carry into up to ~10 ulps of the stored rho E.  Pins: at least 70% of
    the sampled values exact, all within 16 ulps."""
    cfg = tgv.Config(n=256, mode=mode, encoding="offset" if mode == "fp16_fp32" else "plain")
    dt = 0.00125
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    q_in = qa.clone()
    par = tgv.rk_step(cfg, qa, qb, qt, dt, 1)
    q_out = qb if par else qa
    torch.cuda.synchronize()
    wf = window_flow(cfg, half=8)
    rng = np.random.Generator(np.random.PCG64(4242))
    pts = [tuple(int(v) for v in rng.integers(0, cfg.n, size=3)) for _ in range(16)]
    pts += [(0, 0, 0), (255, 255, 255), (128, 0, 255)]
    r0, e0 = (1.0, 1.0 / (cfg.gamma * (cfg.gamma - 1) * cfg.mach ** 2)) \
        if cfg.encoding == "offset" else (0.0, 0.0)
    off = torch.tensor([r0, 0.0, 0.0, 0.0, e0], dtype=torch.float64)
    h = cfg.length / cfg.n
    big = 1.0 / (cfg.gamma * (cfg.gamma - 1) * cfg.mach ** 2) + 1.0 / (cfg.gamma * cfg.mach ** 2)
    arith = 12 * dt * 2.0 ** -24 * torch.tensor([4.0, big + 4, big + 4, big + 4, big + 4],
                                                 dtype=torch.float64) * 1.5 / h
    worst, exact, total = 0.0, 0, 0
    for k, j, i in pts:
        w = decode(cfg, window(q_in, k, j, i, half=8))
        got = decode(cfg, q_out[:, k, j, i].reshape(5, 1, 1, 1)).reshape(5)
        if mode == "fp16_fp32":
            o5 = off.view(5, 1, 1, 1)
            ref = _rk3_step_stored(wf, w, dt, lambda q: (q - o5).half(),
                                   lambda r: r.double() + o5)[:, 8, 8, 8]
            stored = (ref - off).abs()
            # FP16 spacing at the stored magnitude (2^-24 in the subnormal range)
            ulp = torch.exp2(torch.floor(torch.log2(stored.clamp_min(2.0 ** -14))) - 10)
            bound = 16 * ulp
            exact += int((got == ref).sum())
            total += 5
        else:
            ref = oracle.rk3_step(wf, w, dt)[:, 8, 8, 8]
            bound = 3 * 2.0 ** -24 * ((ref - off).abs() + 1e-4) + arith
        worst = max(worst, float(((got - ref).abs() / bound).max()))
        assert bool(((got - ref).abs() <= bound).all()), ((k, j, i), got - ref, bound)
    print(f"\n{mode}: largest error / bound = {worst:.3f}; exact {exact} of {total}")
    if mode == "fp16_fp32":
        assert exact >= 0.7 * total, (exact, total)


def test_full_size_rk_step_sampled_headline_hpsp():
    """The benchmark's headline configuration end to end: one full rk_step at
    256^3 in the HPSP mode (Q FP32, the increment stored in FP16, kept divided
    by dt), at sampled points, against the oracle step on a 16^3 periodic
    window with Q rounded to FP32 and the increment to FP16 where rk_step
    stores them.  FP32 against FP64 arithmetic in the residual may flip the
    FP16 rounding of a stored increment (one FP16 ulp, 2^-11 of it), which the
    stage weight B dt carries into Q; bound per value: three FP32 roundings of
    the stored value, the FP32 arithmetic term of the FP32 mode's bound, and
    one FP16 ulp of the largest stored increment times the sum of B dt."""
    cfg = tgv.Config(n=256, mode="hpsp")
    dt = 0.00125
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    q_in = qa.clone()
    par = tgv.rk_step(cfg, qa, qb, qt, dt, 1)
    q_out = qb if par else qa
    torch.cuda.synchronize()
    wf = window_flow(cfg, half=8)
    rng = np.random.Generator(np.random.PCG64(4343))
    pts = [tuple(int(v) for v in rng.integers(0, cfg.n, size=3)) for _ in range(16)]
    pts += [(0, 0, 0), (255, 255, 255), (128, 0, 255)]
    h = cfg.length / cfg.n
    big = 1.0 / (cfg.gamma * (cfg.gamma - 1) * cfg.mach ** 2) + 1.0 / (cfg.gamma * cfg.mach ** 2)
    arith = 12 * dt * 2.0 ** -24 * torch.tensor([4.0, big + 4, big + 4, big + 4, big + 4],
                                                 dtype=torch.float64) * 1.5 / h
    worst, exact, total = 0.0, 0, 0
    for k, j, i in pts:
        q = decode(cfg, window(q_in, k, j, i, half=8))
        w = torch.zeros_like(q)
        wmax = torch.zeros(5, dtype=torch.float64)
        for st in range(3):
            w = oracle.RK_A[st] * w + oracle.residual(wf, q)
            if st < 2:
                w = w.half().double()
            wmax = torch.maximum(wmax, w[:, 8, 8, 8].abs())
            q = (q + oracle.RK_B[st] * dt * w).float().double()
        ref = q[:, 8, 8, 8]
        got = decode(cfg, q_out[:, k, j, i].reshape(5, 1, 1, 1)).reshape(5)
        bound = (3 * 2.0 ** -24 * (ref.abs() + 1e-4) + arith
                 + sum(oracle.RK_B) * dt * 2.0 ** -10 * wmax)
        exact += int((got == ref).sum())
        total += 5
        worst = max(worst, float(((got - ref).abs() / bound).max()))
        assert bool(((got - ref).abs() <= bound).all()), ((k, j, i), got - ref, bound)
    print(f"\nhpsp: largest error / bound = {worst:.3f}; exact {exact} of {total}")


@pytest.mark.parametrize("split", ["feiereisen", "kgp", "keep"])
@pytest.mark.parametrize("n,tile", [(32, 0), (40, 0), (48, 3)])
def test_study_splits_rhs_and_steps_match_oracle(n, tile, split):
    """The Feiereisen, KGP and KEEP splits of the study (FP64): residual on a
    random state, and 5 RK3 steps."""
    cfg = tgv.Config(n=n, mode="fp64", split=split, mach=0.3, re=100.0, tile=tile)
    flow = oracle_flow(cfg)
    q64 = random_state(cfg, seed=17 + n)
    r = torch.empty(5, n, n, n, dtype=torch.float64, device="cuda")
    tgv.rhs_eval(cfg, encode(cfg, q64), r)
    assert max(max_rel(r.cpu(), oracle.residual(flow, q64))) < 1e-11
    qa = encode(cfg, q64)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, 0.002, 5)
    ref = oracle.run(flow, q64, 0.002, 5)
    assert max(rel_l2((qb if par else qa).cpu(), ref)) < 1e-12


@pytest.mark.parametrize("split", ["feiereisen", "kgp", "keep"])
def test_study_splits_unsupported_in_the_adjoint_and_the_ensemble(split):
    cfg = tgv.Config(n=32, mode="fp64", split=split)
    q = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q)
    lam = torch.zeros(5, 32, 32, 32, dtype=torch.float64, device="cuda")
    with pytest.raises(tgv.TGVError) as ei:
        tgv.rhs_vjp(cfg, q, lam, torch.empty_like(lam))
    assert ei.value.status == tgv._abi.TGV_ERR_UNSUPPORTED
    c32 = cfg.with_(mode="fp32")
    qa = tgv.empty_state(c32)
    with pytest.raises(tgv.TGVError) as ei:
        tgv.Ensemble([c32], [qa], [torch.empty_like(qa)], [tgv.empty_qt(c32)], [0.004])
    assert ei.value.status in (tgv._abi.TGV_ERR_UNSUPPORTED, tgv._abi.TGV_ERR_ARG)


# mode -> bound on max |R - R_oracle| / max |R_oracle| per field, the oracle
# evaluated on the decoded stored state (so only the arithmetic differs):
# FP32 arithmetic 5e-6 (about 80 units of FP32 rounding; measured 2-3e-7),
# FP64 arithmetic 1e-11 (measured 6e-16), FP16 arithmetic 1e-2 (about 20 units
# of FP16 rounding; measured 2.2e-3).
STUDY_MODES = {"fp32": 5e-6, "hpsp": 5e-6, "spdp": 5e-6, "fp32s_fp64c": 1e-11,
               "bf16_fp32": 5e-6, "fp16_fp32": 5e-6, "fp16": 1e-2}


@pytest.mark.parametrize("split", ["feiereisen", "kgp", "keep"])
@pytest.mark.parametrize("mode", list(STUDY_MODES))
def test_study_splits_every_mode_rhs(mode, split):
    """The study's split forms in every precision mode: the residual on a
    random state against the oracle's on the same (decoded) stored state."""
    enc = "offset" if mode in ("bf16_fp32", "fp16_fp32", "fp16") else "plain"
    cfg = tgv.Config(n=32, mode=mode, split=split, mach=0.3, re=100.0, encoding=enc)
    q64 = random_state(cfg, seed=29)
    qs = encode(cfg, q64)
    r = torch.empty(5, 32, 32, 32, dtype=cfg.compute_dtype, device="cuda")
    tgv.rhs_eval(cfg, qs, r)
    ref = oracle.residual(oracle_flow(cfg), decode(cfg, qs))
    err = max(max_rel(r.double().cpu(), ref))
    print(f"\n{mode:12s} {split:10s} max field error {err:.2e}")
    assert err < STUDY_MODES[mode], err
