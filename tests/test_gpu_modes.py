"""Every precision mode against the FP64 oracle: 32^3 Taylor-Green, M = 0.1,
Re = 1600, dt = 0.004, 100 RK3 steps, kinetic energy logged every 10 steps.

Errors reported per mode: relative L2 of rho, of the momentum vector and of
rho E after 100 steps, and the relative error of the dissipation rate
-dK/dt (central differences of the logged K), max over time / max |ref|.
Bounds come from the rounding unit u of the narrowest type a quantity passes
through, times the number of roundings that accumulate (see each entry).
"""
import json
import math

import pytest
import torch

import oracle
import paper_2505_20911_b300 as tgv
from _util import decode, oracle_flow

pytestmark = pytest.mark.gpu

N, DT, STEPS, EVERY = 32, 0.004, 100, 10

# The method's accuracy target for the reduced-precision modes: the relative
# error of the dissipation rate -dK/dt against the FP64 oracle at most 1e-2.
DISS_TARGET = 1e-2

# mode -> (encoding, bound on field errors, bound on dissipation-rate error, kind)
#   kind "target": the mode is offered as meeting DISS_TARGET; its bound is
#     the tighter of DISS_TARGET and the rounding-derived bound below, and the
#     test also asserts DISS_TARGET itself.
#   kind "measured": the mode does not meet DISS_TARGET (Q stored in 16 bits);
#     its bounds are a regression band of about 3x the errors measured on a
#     B300 at this size, not the target (measured: bf16_fp32 fields 8.1e-2,
#     dissipation 1.26; fp16_fp32 2.3e-2, 3.34; fp16 4.1e-2, 0.81).
#   FP32-class arithmetic and Q storage (u = 6e-8): about STEPS * 3 roundings
#     of Q whose effect on the momentum is amplified by the pressure-dominated
#     flux sums (|rho E + p| / |R| ~ 1e2): fields ~1e-5, dissipation rate
#     (a difference of K over 20 steps, K changing by ~1e-5 of itself) ~1e-4.
#   Q stored in 16 bits (bf16 u = 4e-3, fp16 u = 5e-4 on the O(1) momentum):
#     the stage increments B dt R ~ 3e-4 are comparable to half an ulp, so
#     round-to-nearest drops or biases them; the momentum drifts by 1e-2 and
#     the dissipation rate, which lives on those increments, is not resolved.
MODES = {
    "fp64": ("plain", 1e-10, 1e-8, "target"),
    "spdp": ("plain", 5e-6, 1e-4, "target"),
    "fp32s_fp64c": ("plain", 2e-5, 5e-4, "target"),
    "fp32": ("plain", 2e-5, 5e-4, "target"),
    "hpsp": ("plain", 2e-5, 5e-4, "target"),
    "bf16_fp32": ("offset", 2.5e-1, 4.0, "measured"),
    "fp16_fp32": ("offset", 7e-2, 10.0, "measured"),
    "fp16": ("offset", 1.2e-1, 2.5, "measured"),
}


@pytest.fixture(scope="module")
def reference():
    cfg = tgv.Config(n=N, mode="fp64")
    flow = oracle_flow(cfg)
    q, log = oracle.run(flow, oracle.initial_condition(flow), DT, STEPS, log_every=EVERY)
    return q, [d["K"] for _, d in log]


def _run(mode, encoding):
    cfg = tgv.Config(n=N, mode=mode, encoding=encoding)
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    nrec = STEPS // EVERY + 1
    diag = torch.empty(nrec, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    par = tgv.rk_step(cfg, qa, qb, qt, DT, STEPS, EVERY, diag, tgv.empty_workspace(cfg))
    return decode(cfg, qb if par else qa), diag[:, 0].cpu().tolist()


def _dissipation(K):
    return [-(K[i + 1] - K[i - 1]) / (2 * EVERY * DT) for i in range(1, len(K) - 1)]


def mode_errors(mode, encoding, reference):
    q_ref, K_ref = reference
    q, K = _run(mode, encoding)
    nrm = lambda a: float(torch.linalg.vector_norm(a))
    e_rho = nrm(q[0] - q_ref[0]) / nrm(q_ref[0])
    e_mom = nrm(q[1:4] - q_ref[1:4]) / nrm(q_ref[1:4])
    e_E = nrm(q[4] - q_ref[4]) / nrm(q_ref[4])
    # pressure fluctuation: what the low-Mach acoustics see
    flow = oracle_flow(tgv.Config(n=N))
    p, p_ref = oracle.primitives(flow, q)[4], oracle.primitives(flow, q_ref)[4]
    e_p = nrm(p - p_ref) / nrm(p_ref - p_ref.mean())
    eps, eps_ref = _dissipation(K), _dissipation(K_ref)
    e_diss = max(abs(a - b) for a, b in zip(eps, eps_ref)) / max(abs(b) for b in eps_ref)
    return {"rho": e_rho, "mom": e_mom, "rhoE": e_E, "p'": e_p, "diss": e_diss}


@pytest.mark.parametrize("mode", list(MODES))
def test_mode_error_against_oracle(mode, reference):
    enc, bound_field, bound_diss, kind = MODES[mode]
    e = mode_errors(mode, enc, reference)
    print(f"\n{mode:12s} {enc:6s} {kind:8s} " + " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    assert all(math.isfinite(v) for v in e.values()), (mode, e)
    assert max(e["rho"], e["mom"], e["rhoE"]) <= bound_field, (mode, e)
    if kind == "target":
        assert e["diss"] <= min(bound_diss, DISS_TARGET), (mode, e)
    elif bound_diss is not None:
        assert e["diss"] <= bound_diss, (mode, e)


def test_offset_encoding_keeps_the_pressure_fluctuation():
    """At M = 0.1, rho E ~ 178.6 while its fluctuations are O(0.5): plain FP16
    (ulp 0.125 at 178) keeps only a few bits of them, the offset encoding
    (rho E - (rho E)0, ulp ~5e-4) keeps them to ~1e-4.  Pin: the pressure
    fluctuation of the stored initial field, against the oracle's."""
    flow = oracle_flow(tgv.Config(n=N))
    p_ref = oracle.primitives(flow, oracle.initial_condition(flow))[4]
    errs = {}
    for enc in ("plain", "offset"):
        cfg = tgv.Config(n=N, mode="fp16_fp32", encoding=enc)
        q = tgv.empty_state(cfg)
        tgv.tgv_init(cfg, q)
        p = oracle.primitives(flow, decode(cfg, q))[4]
        errs[enc] = float(torch.linalg.vector_norm(p - p_ref)
                          / torch.linalg.vector_norm(p_ref - p_ref.mean()))
    print(f"\npressure-fluctuation error of the stored initial field: {errs}")
    assert errs["offset"] < 2e-3 and errs["offset"] * 50 < errs["plain"], errs
