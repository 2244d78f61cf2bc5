"""Z-slab domain decomposition of the periodic N^3 box (the parallel strategy
of Sec. 4.3: each process owns a block of the grid and exchanges halo points
with its neighbours before every residual evaluation; here the blocks are
slabs of whole z planes, one per GPU, and the halos travel in the storage
type of Q, so reduced-precision storage shrinks the messages as well).

Slab layout: a slab state is 5 fields of (nz + 4) planes of N x N points:
planes 0-1 are ghosts (copies of the two planes below the slab), planes
2 .. nz+1 are the owned planes (global z0 .. z0+nz-1), planes nz+2 .. nz+3
are ghosts (the two planes above).  Two ghost planes match the stencil
radius of the 4th-order operator in z (every term, including the mixed and
dilatation terms of the viscous stress, reaches at most two planes in z).
Qt of a slab holds only the owned planes.

The exchange fills every slab's ghosts from its periodic neighbours:
  ghosts 0-1 of rank r   <- owned planes nz-2, nz-1 of rank r-1 (its top two)
  ghosts nz+2.. of rank r <- owned planes 0, 1 of rank r+1 (its bottom two)
Per field each of these blocks is contiguous, so a message is one field's
two planes; no packing kernel is needed.
"""
from __future__ import annotations

GHOST = 2


def slab_bounds(n: int, world: int, rank: int) -> tuple[int, int]:
    """(z0, nz) of rank's slab: N planes split as evenly as possible, the first
    N % world ranks one plane more.  Every slab needs nz >= GHOST planes (its
    neighbours' ghosts come from it alone)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(n, world)
    nz = base + (1 if rank < extra else 0)
    z0 = rank * base + min(rank, extra)
    if base < GHOST:
        raise ValueError(f"{world} slabs of a {n}-plane grid leave fewer than {GHOST} planes "
                         "in a slab")
    return z0, nz


def mirror_ghosts(q, lower: bool, upper: bool) -> None:
    """Ghosts beyond a mirror face of the symmetric box (slab layout): the
    slab's own two outermost owned planes in reverse order (plane -1 <- 0,
    -2 <- 1 below; N <- N-1, N+1 <- N-2 above), raw - the stage kernel makes
    the mirror's sign change when it reads them."""
    nz = q.shape[1] - 2 * GHOST
    if lower:
        q[:, 0].copy_(q[:, 3])
        q[:, 1].copy_(q[:, 2])
    if upper:
        q[:, nz + 2].copy_(q[:, nz + 1])
        q[:, nz + 3].copy_(q[:, nz])


def ghost_exchange_ops(q, rank: int, world: int, dist, symmetric: bool = False):
    """The point-to-point operations of one ghost exchange of a slab state q
    ((5, nz + 4, N, N), any device), with the buffers they use: the top two
    owned planes of all five fields packed into one block go up, the bottom
    two down, and one block is received from below (the lower ghosts) and one
    from above (the upper ghosts) - four messages per rank instead of one per
    field and direction.  In the symmetric box the first rank has no
    neighbour below and the last none above (mirror faces): those messages
    are left out.  The same order on every rank makes the messages pair up
    correctly also when the two neighbours are the same rank (world = 2: per
    peer, messages match in the order they are posted).
    Returns (ops, recv_lower, recv_upper); a receive buffer is None where no
    message comes."""
    import torch
    nz = q.shape[1] - 2 * GHOST
    lo, hi = (rank - 1) % world, (rank + 1) % world
    has_lo = not (symmetric and rank == 0)
    has_hi = not (symmetric and rank == world - 1)
    ops, recv_lower, recv_upper = [], None, None
    if has_hi:
        ops.append(dist.P2POp(dist.isend, q[:, nz:nz + GHOST].contiguous(), hi))
    if has_lo:
        ops.append(dist.P2POp(dist.isend, q[:, GHOST:2 * GHOST].contiguous(), lo))
        recv_lower = torch.empty_like(q[:, 0:GHOST])
        ops.append(dist.P2POp(dist.irecv, recv_lower, lo))
    if has_hi:
        recv_upper = torch.empty_like(q[:, 0:GHOST])
        ops.append(dist.P2POp(dist.irecv, recv_upper, hi))
    return ops, recv_lower, recv_upper


def exchange_ghosts(q, rank: int, world: int, dist=None, symmetric: bool = False) -> None:
    """Fill the ghost planes of this rank's slab state q from its neighbours
    (torch.distributed point-to-point: NCCL between GPUs, gloo between CPU
    processes) - periodic, or in the symmetric box mirrored at the faces.
    With one rank the slab is the whole box and its ghosts come from its own
    planes (a local copy)."""
    nz = q.shape[1] - 2 * GHOST
    if world == 1:
        if symmetric:
            mirror_ghosts(q, True, True)
        else:
            q[:, 0:GHOST].copy_(q[:, nz:nz + GHOST])
            q[:, nz + GHOST:].copy_(q[:, GHOST:2 * GHOST])
        return
    if dist is None:
        import torch.distributed as dist
    ops, recv_lower, recv_upper = ghost_exchange_ops(q, rank, world, dist, symmetric)
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    if recv_lower is not None:
        q[:, 0:GHOST].copy_(recv_lower)
    if recv_upper is not None:
        q[:, nz + GHOST:].copy_(recv_upper)
    if symmetric:
        mirror_ghosts(q, rank == 0, rank == world - 1)


class SlabDomain:
    """Slabs of one periodic N^3 box advanced with the library's slab stage
    (tgv_slab_substep), the ghosts exchanged before every RK stage.

    local (dist=None): all `slabs` of the box live on the current device and
      exchange by device copies (tgv_slab_exchange_local);
    distributed: this rank owns the single slab slabs[0] = slab_bounds(N,
      world, rank) and exchanges over torch.distributed (NCCL between GPUs).
    """

    def __init__(self, cfg, slabs, rank: int = 0, world: int = 1, dist=None, device=None):
        import torch
        import paper_2505_20911_b300 as tgv
        self.tgv, self.cfg = tgv, cfg
        self.slabs = [tuple(s) for s in slabs]
        self.rank, self.world, self.dist = rank, world, dist
        if dist is not None and len(self.slabs) != 1:
            raise ValueError("a distributed rank owns exactly one slab")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.q = [[tgv.empty_slab_state(cfg, nz, dev), tgv.empty_slab_state(cfg, nz, dev)]
                  for _, nz in self.slabs]
        self.qt = [tgv.empty_slab_qt(cfg, nz, dev) for _, nz in self.slabs]
        self.ws = tgv.empty_workspace(cfg, dev)
        self.cur = 0

    def init(self, stream=None) -> None:
        for (z0, nz), q in zip(self.slabs, self.q):
            self.tgv.tgv_slab_init(self.cfg, z0, nz, q[0], stream)
        self.cur = 0

    def load(self, full) -> None:
        """Copy the owned planes from a whole-box state (5, N, N, N) on the device."""
        for (z0, nz), q in zip(self.slabs, self.q):
            q[0][:, GHOST:GHOST + nz].copy_(full[:, z0:z0 + nz])
        self.cur = 0

    def state(self, r: int = 0):
        """The current state of slab r (slab layout)."""
        return self.q[r][self.cur]

    def owned(self, r: int = 0):
        _, nz = self.slabs[r]
        return self.state(r)[:, GHOST:GHOST + nz]

    def exchange(self, stream=None) -> None:
        if self.dist is None:
            self.tgv.tgv_slab_exchange_local(self.cfg, self.slabs,
                                             [q[self.cur] for q in self.q], stream)
        else:
            exchange_ghosts(self.q[0][self.cur], self.rank, self.world, self.dist,
                            bool(self.cfg.symmetric))

    def step(self, dt: float, nsteps: int = 1, diag=None, stream=None) -> None:
        """nsteps RK3 steps; diag (optional device double[TGV_DIAG_COUNT]) receives
        the diagnostics of the state at the start of the last step, summed over
        this process's slabs (the whole box locally; this rank's share when
        distributed, to be all-reduced)."""
        import torch
        for m in range(nsteps):
            want = diag is not None and m == nsteps - 1
            if want:
                diag.zero_()
                part = torch.empty_like(diag)
            for i in range(3):
                self.exchange(stream)
                for r, (z0, nz) in enumerate(self.slabs):
                    q = self.q[r]
                    d = part if (want and i == 0) else None
                    self.tgv.tgv_slab_substep(self.cfg, z0, nz, q[self.cur], q[self.cur ^ 1],
                                              self.qt[r], i, dt, d, self.ws if d is not None
                                              else None, stream)
                    if d is not None:
                        diag.add_(part)
                self.cur ^= 1
