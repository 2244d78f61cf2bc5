"""The z-slab path on one GPU: P slabs of one periodic (or symmetric) box on
the same device, ghosts exchanged by a copy kernel before every stage, equal the
whole-box rk_step bit for bit on every owned plane (the stage arithmetic of
a point does not depend on which CTA or slab computes it), and their
diagnostics contributions add up to the whole box's."""
import pytest
import torch

import paper_2505_20911_b300 as tgv
from paper_2505_20911_b300 import slab
from _util import random_state, encode

pytestmark = pytest.mark.gpu


def _whole_box(cfg, q0, dt, steps):
    qa = q0.clone()
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, dt, steps)
    return qb if par else qa


@pytest.mark.parametrize("mode,n,world", [("fp32", 32, 2), ("hpsp", 40, 3), ("fp64", 32, 4),
                                          ("fp16_fp32", 48, 2), ("spdp", 32, 3)])
def test_slabs_on_one_device_equal_the_whole_box(mode, n, world):
    cfg = tgv.Config(n=n, mode=mode, encoding="offset" if mode == "fp16_fp32" else "plain")
    q0 = encode(cfg, random_state(cfg, 5))
    dt = 0.5 * tgv.tgv_dt_max(cfg)
    ref = _whole_box(cfg, q0, dt, 3)
    spans = [slab.slab_bounds(n, world, r) for r in range(world)]
    dom = slab.SlabDomain(cfg, spans)
    dom.load(q0)
    dom.step(dt, 3)
    torch.cuda.synchronize()
    for r, (z0, nz) in enumerate(spans):
        assert torch.equal(dom.owned(r), ref[:, z0:z0 + nz]), (mode, r)


def test_slab_initial_condition_and_diagnostics_add_up():
    n, world = 32, 4
    cfg = tgv.Config(n=n, mode="fp64")
    full = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, full)
    spans = [slab.slab_bounds(n, world, r) for r in range(world)]
    dom = slab.SlabDomain(cfg, spans)
    dom.init()
    for r, (z0, nz) in enumerate(spans):
        assert torch.equal(dom.owned(r), full[:, z0:z0 + nz])
    diag = torch.empty(tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    dom.step(0.004, 1, diag=diag)
    ref = tgv.diagnostics(cfg, full)
    got = dict(zip(tgv.DIAG_NAMES, diag.cpu().tolist()))
    for k in ("K", "K_rho", "enstrophy", "eps_S", "rho", "rho_E"):
        assert got[k] == pytest.approx(ref[k], rel=1e-13, abs=1e-15), k
    assert got["nonfinite"] == 0.0


def test_one_slab_wraps_onto_itself():
    cfg = tgv.Config(n=32, mode="fp32")
    q0 = encode(cfg, random_state(cfg, 9))
    dt = 0.004
    ref = _whole_box(cfg, q0, dt, 2)
    dom = slab.SlabDomain(cfg, [(0, 32)])
    dom.load(q0)
    dom.step(dt, 2)
    assert torch.equal(dom.owned(0), ref)


@pytest.mark.parametrize("mode,world", [("fp64", 2), ("hpsp", 3), ("fp32", 4), ("fp16", 2)])
def test_symmetric_box_slabs_equal_the_whole_box(mode, world):
    """The symmetric box (TGSym: mirror planes on every face) in z-slabs: the
    first and last slabs' outer ghosts are mirror images of their own planes,
    the inner ones come from the neighbours; 5 steps equal the whole-box
    rk_step bit for bit."""
    n = 32
    cfg = tgv.Config(n=n, mode=mode, length=3.141592653589793, symmetric=True, mach=0.5,
                     re=800.0, encoding="offset" if mode == "fp16" else "plain")
    q0 = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q0)
    dt = 0.0025
    ref = _whole_box(cfg, q0, dt, 5)
    spans = [slab.slab_bounds(n, world, r) for r in range(world)]
    dom = slab.SlabDomain(cfg, spans)
    dom.init()
    for r, (z0, nz) in enumerate(spans):
        assert torch.equal(dom.owned(r), q0[:, z0:z0 + nz]), r    # the slab initial condition
    dom.step(dt, 5)
    torch.cuda.synchronize()
    for r, (z0, nz) in enumerate(spans):
        assert torch.equal(dom.owned(r), ref[:, z0:z0 + nz]), (mode, r)


def test_slab_arguments_are_validated():
    cfg = tgv.Config(n=32, mode="fp32")
    assert tgv.tgv_slab_state_bytes(cfg, 0, 1) == 0           # fewer than 2 owned planes
    assert tgv.tgv_slab_state_bytes(cfg, 30, 4) == 0          # beyond the box
    assert tgv.tgv_slab_state_bytes(cfg.with_(symmetric=True, length=3.14159), 0, 8) > 0
    q = tgv.empty_slab_state(cfg, 16)
    with pytest.raises(tgv.TGVError):                         # slabs that do not tile [0, N)
        tgv.tgv_slab_exchange_local(cfg, [(0, 16), (20, 12)], [q, tgv.empty_slab_state(cfg, 12)])
