"""Inviscid Taylor-Green runs (the split-form study of Sec. 4.2: 64^3, M = 0.4,
dt = 0.004, viscous terms off) and the non-finite stop of rk_step.

The paper reports that the plain divergence form diverges quickly while the
quadratic split forms (Blaisdell and Feiereisen among them) keep the kinetic
energy near its initial value much longer, in double and in half-single
precision alike.
It also reports that the cubic KGP and KEEP splits stay stable up to t = 20.
Checked here: the Blaisdell and Feiereisen forms keep K/K0 within 1e-2 of 1
at least as long as the divergence form does, KGP and KEEP stay finite to t = 20 and keep K/K0
within 1e-2 at least as long as Blaisdell, in FP64 and in the Q FP32 / Qt FP16
mode; and the first non-finite state stops rk_step with TGV_ERR_NONFINITE.
"""
import math

import pytest
import torch

import paper_2505_20911_b300 as tgv
from paper_2505_20911_b300 import _abi

pytestmark = pytest.mark.gpu

N, M, DT, T_END, EVERY = 64, 0.4, 0.004, 20.0, 25


def _history(mode, split):
    """K/K0 every EVERY steps until T_END or the first non-finite state."""
    cfg = tgv.Config(n=N, mode=mode, mach=M, mu=0.0, split=split, check_finite=True)
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    nsteps = int(round(T_END / DT))
    diag = torch.full((nsteps // EVERY + 1, tgv.TGV_DIAG_COUNT), float("nan"),
                      dtype=torch.float64, device="cuda")
    blew_up = False
    try:
        tgv.rk_step(cfg, qa, qb, qt, DT, nsteps, EVERY, diag, tgv.empty_workspace(cfg))
    except tgv.TGVError as e:
        assert e.status == _abi.TGV_ERR_NONFINITE, e
        blew_up = True
    K = diag[:, 0].cpu().tolist()
    K0 = K[0]
    ratio = [k / K0 for k in K if math.isfinite(k)]
    return ratio, blew_up


def _time_within(ratio, tol=1e-2):
    """Time until K/K0 first leaves [1 - tol, 1 + tol]."""
    for i, r in enumerate(ratio):
        if abs(r - 1.0) > tol:
            return i * EVERY * DT
    return len(ratio) * EVERY * DT


@pytest.mark.parametrize("mode", ["fp64", "hpsp"])
def test_split_forms_in_the_inviscid_limit(mode):
    r_b, nan_b = _history(mode, "blaisdell")
    r_d, nan_d = _history(mode, "divergence")
    r_k, nan_k = _history(mode, "kgp")
    r_e, nan_e = _history(mode, "keep")
    r_f, nan_f = _history(mode, "feiereisen")
    t_b, t_d, t_k = _time_within(r_b), _time_within(r_d), _time_within(r_k)
    t_e, t_f = _time_within(r_e), _time_within(r_f)
    print(f"\n{mode}: K/K0 within 1e-2 until t = {t_d:.2f} divergence (non-finite {nan_d}), "
          f"{t_f:.2f} Feiereisen (non-finite {nan_f}), "
          f"{t_b:.2f} Blaisdell (non-finite {nan_b}), {t_k:.2f} KGP (non-finite {nan_k}), "
          f"{t_e:.2f} KEEP (non-finite {nan_e}); K/K0 at the end: Feiereisen {r_f[-1]:.4f}, "
          f"Blaisdell {r_b[-1]:.4f}, KGP {r_k[-1]:.4f}, KEEP {r_e[-1]:.4f}")
    assert t_b >= t_d and t_f >= t_d
    assert not nan_k and t_k >= t_b
    assert not nan_e and t_e >= t_b
    assert r_b[int(1.0 / (EVERY * DT))] == pytest.approx(1.0, abs=2e-3)  # t = 1


def test_nonfinite_state_stops_rk_step():
    cfg = tgv.Config(n=32, mode="fp32", check_finite=True)
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    qa[1, 5, 6, 7] = float("nan")          # the failure is planted in the input data
    diag = torch.zeros(11, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    with pytest.raises(tgv.TGVError) as ei:
        tgv.rk_step(cfg, qa, qb, qt, 0.004, 10, 1, diag, tgv.empty_workspace(cfg))
    assert ei.value.status == _abi.TGV_ERR_NONFINITE
    assert float(diag[0, 9]) >= 1.0         # the first record counted the bad point
    # without the flag the run completes and the records carry the count
    cfg2 = cfg.with_(check_finite=False)
    tgv.rk_step(cfg2, qa, qb, qt, 0.004, 2, 1, diag, tgv.empty_workspace(cfg2))
    assert float(diag[0, 9]) >= 1.0
