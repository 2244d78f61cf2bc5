"""rk_step is stream-ordered and never synchronises the host unless asked to
(diagnostics with TGV_FLAG_CHECK_FINITE), so a caller can capture it into a
CUDA graph: replays give the same state as direct calls, bit for bit."""
import pytest
import torch

import paper_2505_20911_b300 as tgv

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,n", [("fp32", 32), ("fp16_fp32", 48), ("fp64", 16)])
def test_rk_step_replays_from_a_cuda_graph(mode, n):
    cfg = tgv.Config(n=n, mode=mode, encoding="offset" if mode == "fp16_fp32" else "plain")
    dt = 0.5 * tgv.tgv_dt_max(cfg)
    q0 = tgv.empty_state(cfg)
    tgv.tgv_init(cfg, q0)

    # direct: 30 steps
    qa, qb, qt = q0.clone(), torch.empty_like(q0), tgv.empty_qt(cfg)
    par = tgv.rk_step(cfg, qa, qb, qt, dt, 30)
    direct = (qb if par else qa).clone()

    # graph: 10 steps per replay (an even count, so each replay ends in ga)
    ga, gb, gt = q0.clone(), torch.empty_like(q0), tgv.empty_qt(cfg)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):          # warm the library's per-device caches
        tgv.rk_step(cfg, gb.copy_(q0), ga, gt, dt, 2)
    torch.cuda.current_stream().wait_stream(side)
    ga.copy_(q0)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        assert tgv.rk_step(cfg, ga, gb, gt, dt, 10) == 0
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ga, direct)
