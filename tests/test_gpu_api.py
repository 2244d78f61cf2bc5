"""The host-buffer entry point and the workspace / argument errors of the C ABI
on a device."""
import pytest
import torch

import paper_2505_20911_b300 as tgv
from paper_2505_20911_b300 import _abi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["fp64", "fp16_fp32"])
def test_run_host_matches_device_path_bitwise(mode):
    cfg = tgv.Config(n=48, mode=mode, encoding="offset" if mode == "fp16_fp32" else "plain")
    q0 = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q0)
    # device path
    qa, qb, qt = q0.clone(), torch.empty_like(q0), tgv.empty_qt(cfg)
    diag = torch.empty(3, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    par = tgv.rk_step(cfg, qa, qb, qt, 0.004, 10, 5, diag, tgv.empty_workspace(cfg))
    ref = (qb if par else qa).cpu()
    # host path: pinned host in/out, device workspace from the caller
    h_in = q0.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_host = torch.empty(3 * tgv.TGV_DIAG_COUNT, dtype=torch.float64).pin_memory()
    ws = torch.empty(tgv.tgv_run_host_workspace_bytes(cfg, 10, 5), dtype=torch.uint8, device="cuda")
    tgv.tgv_run_host(cfg, h_in, h_out, 0.004, 10, 5, d_host, ws)
    assert torch.equal(h_out, ref)
    assert torch.equal(d_host.view(3, -1), diag.cpu())


@pytest.mark.parametrize("mode", ["fp32", "fp16_fp32"])
@pytest.mark.parametrize("count", [1, 2, 5])
def test_run_host_stream_matches_single_calls_bitwise(mode, count):
    """The pipelined host call: each of `count` different states (the TGV
    field scaled by a different factor) comes back exactly as from
    tgv_run_host, records included, with the copies on a second stream."""
    cfg = tgv.Config(n=32, mode=mode, encoding="offset" if mode == "fp16_fp32" else "plain")
    q0 = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q0)
    base = q0.cpu()
    ins = []
    for i in range(count):
        q = base.clone()
        q[1:4] = (q[1:4].float() * (1.0 - 0.1 * i)).to(q.dtype)  # slower vortices
        ins.append(q.pin_memory())
    outs = [torch.empty_like(q).pin_memory() for q in ins]
    nsteps, every = 6, 3
    nrec = nsteps // every + 1
    d_host = torch.zeros(count * nrec * tgv.TGV_DIAG_COUNT, dtype=torch.float64).pin_memory()
    ws = torch.empty(tgv.tgv_run_host_stream_workspace_bytes(cfg, nsteps, every),
                     dtype=torch.uint8, device="cuda")
    tgv.tgv_run_host_stream(cfg, ins, outs, 0.004, nsteps, every, d_host, ws,
                            copy_stream=torch.cuda.Stream())
    ws1 = torch.empty(tgv.tgv_run_host_workspace_bytes(cfg, nsteps, every), dtype=torch.uint8,
                      device="cuda")
    for i in range(count):
        ref = torch.empty_like(ins[i]).pin_memory()
        d1 = torch.empty(nrec * tgv.TGV_DIAG_COUNT, dtype=torch.float64).pin_memory()
        tgv.tgv_run_host(cfg, ins[i], ref, 0.004, nsteps, every, d1, ws1)
        assert torch.equal(outs[i], ref), i
        assert torch.equal(d_host.view(count, -1)[i], d1), i


def test_run_host_stream_argument_errors():
    cfg = tgv.Config(n=32)
    h = torch.empty((5, 32, 32, 32), dtype=torch.float64).pin_memory()
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(tgv.TGVError) as ei:
        tgv.tgv_run_host_stream(cfg, [h], [h], 0.004, 2, 0, None, small,
                                copy_stream=torch.cuda.Stream())
    assert ei.value.status == _abi.TGV_ERR_WORKSPACE
    ws = torch.empty(tgv.tgv_run_host_stream_workspace_bytes(cfg, 2, 0), dtype=torch.uint8,
                     device="cuda")
    tgv.tgv_run_host_stream(cfg, [], [], 0.004, 2, 0, None, ws, copy_stream=torch.cuda.Stream())


def test_workspace_errors():
    cfg = tgv.Config(n=32)
    q = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q)
    out = torch.empty(tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(tgv.TGVError) as ei:
        tgv.diagnostics_reduce(cfg, q, out, small)
    assert ei.value.status == _abi.TGV_ERR_WORKSPACE
    qb, qt = torch.empty_like(q), tgv.empty_qt(cfg)
    diag = torch.empty(2, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    with pytest.raises(tgv.TGVError) as ei:
        tgv.rk_step(cfg, q, qb, qt, 0.004, 1, 1, diag, small)
    assert ei.value.status == _abi.TGV_ERR_WORKSPACE
    with pytest.raises(tgv.TGVError) as ei:
        tgv.rk_step(cfg, q, qb, qt, 0.05, 1)           # above the stability limit
    assert ei.value.status == _abi.TGV_ERR_UNSTABLE_DT
    tgv.rk_step(cfg.with_(allow_unstable_dt=True), q, qb, qt, 0.02, 1)  # allowed when asked


def test_resume_from_a_checkpoint_is_bit_exact(tmp_path):
    """6 steps in one go equal 3 steps, save, load, 3 more steps (the RK
    increment restarts every step, so Q alone carries the run)."""
    import os
    from paper_2505_20911_b300 import checkpoint
    cfg = tgv.Config(n=32, mode="hpsp")
    dt = 0.004
    qa = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, qa)
    q0 = qa.clone()
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, dt, 6)
    straight = (qb if par else qa).clone()
    qa.copy_(q0)
    par = tgv.rk_step(cfg, qa, qb, qt, dt, 3)
    path = os.path.join(tmp_path, "mid.tgvq")
    checkpoint.save_state(path, cfg, qb if par else qa, step=3, time=3 * dt)
    cfg2, q3, step, t = checkpoint.load_state(path)
    assert cfg2 == cfg and step == 3
    qa2 = q3.contiguous()
    qb2, qt2 = torch.empty_like(qa2), tgv.empty_qt(cfg2)
    par = tgv.rk_step(cfg2, qa2, qb2, qt2, dt, 3)
    assert torch.equal(qb2 if par else qa2, straight)
