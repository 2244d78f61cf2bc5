"""The z-slab decomposition's host logic (paper_2505_20911_b300.slab: the slab
bounds and the ghost exchange over torch.distributed, periodic and in the
symmetric box) on CPU ranks with the gloo backend, world sizes 2 and 4.  Each rank advances its slab with the FP64
oracle on the slab plus its ghost planes; after every exchange the owned
planes see exactly the neighbours the whole periodic box gives them, so the
gathered slabs equal the single-domain oracle run bit for bit."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

N, STEPS, DT = 16, 3, 0.004


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _state():
    import oracle
    import tgv_inputs
    flow = oracle.Flow(n=N)
    rho, u, v, w, dp = (torch.from_numpy(a) for a in tgv_inputs.random_flow_fields(N, 11))
    return flow, oracle.conserved(flow, rho, u, v, w, 1.0 / (flow.gamma * flow.mach ** 2) + dp)


def _worker(rank, world, port, out):
    import oracle
    from paper_2505_20911_b300 import slab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        flow, q = _state()
        z0, nz = slab.slab_bounds(N, world, rank)
        g = slab.GHOST
        qs = torch.full((5, nz + 2 * g, N, N), float("nan"), dtype=torch.float64)
        qs[:, g:g + nz] = q[:, z0:z0 + nz]
        for _ in range(STEPS):
            qt = torch.zeros_like(qs)
            for i in range(3):
                slab.exchange_ghosts(qs, rank, world, dist)
                qs, qt = oracle.rk_substep(flow, qs, qt, i, DT)
        parts = [None] * world
        dist.all_gather_object(parts, (z0, qs[:, g:g + nz].clone()))
        if rank == 0:
            full = torch.empty_like(q)
            for zz, part in parts:
                full[:, zz:zz + part.shape[1]] = part
            out["slabs"] = full
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slabs_over_gloo_ranks_equal_the_single_domain_oracle(world):
    import oracle
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    flow, q = _state()
    ref = oracle.run(flow, q, DT, STEPS)
    assert torch.equal(out["slabs"], ref)


def test_slab_bounds_cover_the_grid_once():
    from paper_2505_20911_b300 import slab
    for n, world in ((16, 2), (16, 3), (512, 8), (10, 4), (256, 7)):
        spans = [slab.slab_bounds(n, world, r) for r in range(world)]
        assert spans[0][0] == 0
        for (a, na), (b, _) in zip(spans, spans[1:]):
            assert a + na == b
        assert spans[-1][0] + spans[-1][1] == n
        assert max(s[1] for s in spans) - min(s[1] for s in spans) <= 1
    with pytest.raises(ValueError):
        slab.slab_bounds(8, 5, 0)       # slabs of one plane cannot feed two ghost planes


def test_single_rank_ghosts_are_the_periodic_wrap():
    from paper_2505_20911_b300 import slab
    q = torch.arange(5 * 8 * 2 * 2, dtype=torch.float64).reshape(5, 8, 2, 2)
    qs = torch.zeros(5, 12, 2, 2, dtype=torch.float64)
    qs[:, 2:10] = q
    slab.exchange_ghosts(qs, 0, 1)
    assert torch.equal(qs[:, 0:2], q[:, 6:8]) and torch.equal(qs[:, 10:12], q[:, 0:2])


def _mirror_worker(rank, world, port, out):
    from paper_2505_20911_b300 import slab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = torch.arange(5 * N * 3 * 2, dtype=torch.float64).reshape(5, N, 3, 2)
        z0, nz = slab.slab_bounds(N, world, rank)
        qs = torch.full((5, nz + 4, 3, 2), float("nan"), dtype=torch.float64)
        qs[:, 2:2 + nz] = full[:, z0:z0 + nz]
        slab.exchange_ghosts(qs, rank, world, dist, symmetric=True)
        parts = [None] * world
        dist.all_gather_object(parts, (z0, nz, qs))
        if rank == 0:
            out["parts"] = parts
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 4])
def test_symmetric_box_ghost_exchange(world):
    """In the symmetric box the first rank's lower and the last rank's upper
    ghosts are the mirror images of their own planes (global plane -1 <- 0,
    -2 <- 1, N <- N-1, N+1 <- N-2, raw values); every inner ghost is the
    neighbour's plane, exchanged over gloo ranks."""
    from paper_2505_20911_b300 import slab
    full = torch.arange(5 * N * 3 * 2, dtype=torch.float64).reshape(5, N, 3, 2)
    # the whole box's z planes extended by its mirror images
    ext = torch.cat([full[:, 1:2], full[:, 0:1], full, full[:, N - 1:N], full[:, N - 2:N - 1]], 1)
    if world == 1:
        qs = torch.full((5, N + 4, 3, 2), float("nan"), dtype=torch.float64)
        qs[:, 2:2 + N] = full
        slab.exchange_ghosts(qs, 0, 1, symmetric=True)
        assert torch.equal(qs, ext)
        return
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_mirror_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for z0, nz, qs in out["parts"]:
        assert torch.equal(qs, ext[:, z0:z0 + nz + 4]), z0
