"""The batched ensemble equals each instance run alone (bit for bit, same tile
and z chunk), on a small mixed ensemble and on the 48-instance workload
(12 each of 32^3, 48^3, 64^3, 96^3, seeded Re and M, FP32, 500 steps)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_20911_b300 as tgv
from _util import decode, oracle_flow, rel_l2

pytestmark = pytest.mark.gpu


def _alloc(cfgs):
    qa, qb, qt = [], [], []
    for c in cfgs:
        q = tgv.empty_state(c)
        tgv.tgv_init(c, q)
        qa.append(q)
        qb.append(torch.empty_like(q))
        qt.append(tgv.empty_qt(c))
    return qa, qb, qt


def _solo(cfg, dt, nsteps, tile, zc):
    c = cfg.with_(tile=tile, zchunk=min(cfg.n, zc))
    qa = tgv.empty_state(c)
    tgv.tgv_init(c, qa)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(c)
    par = tgv.rk_step(c, qa, qb, qt, dt, nsteps)
    return qb if par else qa


def test_small_mixed_ensemble_matches_solo_runs():
    cfgs = [tgv.Config(n=n, mode="fp32", re=re, mach=m)
            for n, re, m in ((32, 400.0, 0.1), (48, 800.0, 0.2), (64, 1600.0, 0.1),
                             (32, 3200.0, 0.2), (48, 1600.0, 0.1), (64, 400.0, 0.2))]
    dts = [min(0.004, 0.8 * tgv.tgv_dt_max(c)) for c in cfgs]
    qa, qb, qt = _alloc(cfgs)
    ens = tgv.Ensemble(cfgs, qa, qb, qt, dts, steps_per_graph=4)
    info = ens.info()
    ens.run(2)
    torch.cuda.synchronize()
    for i, c in enumerate(cfgs):
        ref = _solo(c, dts[i], 8, info["tile"], info["zchunk_target"])
        assert torch.equal(qa[i], ref), i
    ens.close()


def test_ensemble_pinned_tile_and_zchunk():
    cfgs = [tgv.Config(n=32, mode="fp32", tile=3, zchunk=12), tgv.Config(n=48, mode="fp32")]
    dts = [0.003, 0.003]
    qa, qb, qt = _alloc(cfgs)
    ens = tgv.Ensemble(cfgs, qa, qb, qt, dts, steps_per_graph=2)
    info = ens.info()
    assert info["tile"] == 3 and info["zchunk_target"] == 12
    ens.run(3)
    torch.cuda.synchronize()
    for i, c in enumerate(cfgs):
        assert torch.equal(qa[i], _solo(c.with_(tile=0, zchunk=0), dts[i], 6, 3, 12))
    ens.close()


def test_ensemble_48_instances_500_steps():
    cfgs, dts = tgv.ensemble_instances()
    assert len(cfgs) == 48 and sum(c.n ** 3 for c in cfgs) == 15482880
    qa, qb, qt = _alloc(cfgs)
    ens = tgv.Ensemble(cfgs, qa, qb, qt, dts, steps_per_graph=10)
    info = ens.info()
    ens.run(50)
    torch.cuda.synchronize()
    for i, c in enumerate(cfgs):
        assert bool(torch.isfinite(qa[i]).all()), i
        assert torch.equal(qa[i], _solo(c, dts[i], 500, info["tile"], info["zchunk_target"])), i
    ens.close()


def test_ensemble_instance_matches_oracle_in_fp32_tolerance():
    """One 32^3 member after 20 steps against the FP64 oracle.  FP32 rounding
    (2^-24) of the state and of the pressure-dominated flux sums leaves a
    relative L2 error of order 1e-6 in rho, rho E and the momentum vector
    (measured with the momentum's own norm: w starts at zero, so its
    component-wise relative error is meaningless)."""
    cfgs = [tgv.Config(n=32, mode="fp32", re=800.0, mach=0.2),
            tgv.Config(n=48, mode="fp32", re=1600.0, mach=0.1)]
    dts = [0.004, 0.004]
    qa, qb, qt = _alloc(cfgs)
    ens = tgv.Ensemble(cfgs, qa, qb, qt, dts, steps_per_graph=10)
    ens.run(2)
    torch.cuda.synchronize()
    flow = oracle_flow(cfgs[0])
    ref = oracle.run(flow, oracle.initial_condition(flow), 0.004, 20)
    got = decode(cfgs[0], qa[0])
    err = rel_l2(got, ref)
    mom = float(torch.linalg.vector_norm(got[1:4] - ref[1:4]) / torch.linalg.vector_norm(ref[1:4]))
    assert mom < 1e-5 and err[0] < 1e-6 and err[4] < 1e-6, (mom, err)
    ens.close()


@pytest.mark.parametrize("mode,enc", [("hpsp", "plain"), ("fp16_fp32", "offset"),
                                      ("fp16", "offset"), ("spdp", "plain"), ("fp64", "plain"),
                                      ("hpsp", "offset"), ("fp32", "offset")])
def test_ensemble_in_every_precision_mode_matches_solo_runs(mode, enc):
    """The ensemble in the other precision modes (one mode per ensemble): each
    instance equals the single-instance rk_step with the ensemble's tile and
    z chunk, bit for bit.  The ensemble's kernel reads the RK flags at run
    time, rk_step's stages have them built in; FP32 storage with FP32
    arithmetic and the offset encoding takes rk_step's runtime-flag kernel
    (its built-in flags assume the plain encoding)."""
    cfgs = [tgv.Config(n=n, mode=mode, re=re, mach=m, encoding=enc)
            for n, re, m in ((32, 400.0, 0.1), (48, 800.0, 0.2), (40, 1600.0, 0.1))]
    dts = [min(0.004, 0.8 * tgv.tgv_dt_max(c)) for c in cfgs]
    qa, qb, qt = _alloc(cfgs)
    ens = tgv.Ensemble(cfgs, qa, qb, qt, dts, steps_per_graph=2)
    info = ens.info()
    ens.run(2)
    torch.cuda.synchronize()
    for i, c in enumerate(cfgs):
        assert torch.equal(qa[i], _solo(c, dts[i], 4, info["tile"], info["zchunk_target"])), i
    ens.close()


def test_ensemble_refuses_mixed_precision_modes():
    cfgs = [tgv.Config(n=32, mode="fp32"), tgv.Config(n=32, mode="hpsp")]
    qa, qb, qt = _alloc(cfgs)
    with pytest.raises(tgv.TGVError) as ei:
        tgv.Ensemble(cfgs, qa, qb, qt, [0.004, 0.004])
    assert ei.value.status == tgv._abi.TGV_ERR_ARG
