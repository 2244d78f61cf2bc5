"""The symmetric box (TGSym: [0, pi]^3, mirror planes, cell-centred) on the GPU
against the oracle, and against one octant of the periodic 2N^3 GPU run."""
import math

import pytest
import torch

import oracle
import paper_2505_20911_b300 as tgv
from _util import decode, encode, max_rel, oracle_flow, random_state, rel_l2

pytestmark = pytest.mark.gpu


def _cfg(n, **kw):
    kw.setdefault("mode", "fp64")
    return tgv.Config(n=n, length=math.pi, symmetric=True, mach=0.5, re=800.0, **kw)


@pytest.mark.parametrize("n,tile", [(32, 0), (40, 1), (48, 3)])
def test_symmetric_rhs_matches_oracle(n, tile):
    cfg = _cfg(n, tile=tile)
    flow = oracle_flow(cfg)
    for q64 in (oracle.initial_condition(flow), random_state(cfg, seed=n)):
        r = torch.empty(5, n, n, n, dtype=torch.float64, device="cuda")
        tgv.rhs_eval(cfg, encode(cfg, q64), r)
        assert max(max_rel(r.cpu(), oracle.residual(flow, q64))) < 1e-11


def test_symmetric_init_steps_and_diagnostics_match_oracle():
    cfg = _cfg(32)
    flow = oracle_flow(cfg)
    qa = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, qa)
    ref0 = oracle.initial_condition(flow)
    assert max(max_rel(qa.cpu(), ref0)[:3] + max_rel(qa.cpu(), ref0)[4:]) < 1e-14
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    diag = torch.empty(3, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    par = tgv.rk_step(cfg, qa, qb, qt, 0.0025, 10, 5, diag, tgv.empty_workspace(cfg))
    ref, log = oracle.run(flow, ref0, 0.0025, 10, log_every=5)
    assert max(rel_l2((qb if par else qa).cpu(), ref)) < 1e-12
    d = diag.cpu()
    for rec, (_, dref) in enumerate(log):
        for m, name in enumerate(tgv.DIAG_NAMES):
            assert abs(float(d[rec, m]) - dref[name]) <= 1e-12 * abs(dref[name]) + 1e-15, name


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_symmetric_box_is_one_octant_of_the_periodic_run(mode):
    n = 32
    cs = _cfg(n, mode=mode)
    cp = tgv.Config(n=2 * n, mode=mode, cell_centered=True, mach=0.5, re=800.0)
    out = []
    for cfg in (cs, cp):
        qa = tgv.empty_state(cfg)
        tgv.tgv_init(cfg, qa)
        qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
        par = tgv.rk_step(cfg, qa, qb, qt, 0.0025, 20)
        out.append((qb if par else qa).double().cpu())
    tol = 1e-12 if mode == "fp64" else 2e-5
    assert max(rel_l2(out[0], out[1][:, :n, :n, :n])) < tol


@pytest.mark.parametrize("split", ["kgp", "keep", "feiereisen", "divergence"])
def test_symmetric_box_with_other_split_forms(split):
    """The mirror ghosts are independent of the convective split: the KGP and
    divergence forms in the symmetric box against the oracle (FP64)."""
    cfg = _cfg(32, split=split)
    flow = oracle_flow(cfg)
    q64 = random_state(cfg, seed=77)
    r = torch.empty(5, 32, 32, 32, dtype=torch.float64, device="cuda")
    tgv.rhs_eval(cfg, encode(cfg, q64), r)
    assert max(max_rel(r.cpu(), oracle.residual(flow, q64))) < 1e-11
    qa = encode(cfg, oracle.initial_condition(flow))
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, 0.0025, 5)
    ref = oracle.run(flow, oracle.initial_condition(flow), 0.0025, 5)
    assert max(rel_l2((qb if par else qa).cpu(), ref)) < 1e-12


@pytest.mark.parametrize("mode", ["fp32", "hpsp", "fp16_fp32"])
def test_symmetric_box_reduced_precision_modes(mode):
    """The TGSym runs of the benchmark's modes: 10 steps at 32^3 against the
    FP64 oracle, within each mode's rounding (FP32 compute: 1e-5 of each field;
    FP16 storage: the field bound of the 32^3 mode test)."""
    cfg = _cfg(32, mode=mode, encoding="offset" if mode == "fp16_fp32" else "plain")
    flow = oracle_flow(cfg)
    qa = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, qa)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, 0.0025, 10)
    ref = oracle.run(flow, oracle.initial_condition(flow), 0.0025, 10)
    q = decode(cfg, qb if par else qa)
    nrm = lambda a: float(torch.linalg.vector_norm(a))
    err = [nrm(q[0] - ref[0]) / nrm(ref[0]), nrm(q[1:4] - ref[1:4]) / nrm(ref[1:4]),
           nrm(q[4] - ref[4]) / nrm(ref[4])]      # rho, momentum vector, rho E
    assert max(err) < (5e-2 if mode == "fp16_fp32" else 1e-5), err
