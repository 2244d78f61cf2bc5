"""Helpers shared by the tests: build seeded states with the oracle and move
them to the device in a precision mode's storage type."""
import math

import torch

import oracle
import tgv_inputs
import paper_2505_20911_b300 as tgv


def oracle_flow(cfg: tgv.Config) -> oracle.Flow:
    return oracle.Flow(n=cfg.n, gamma=cfg.gamma, mach=cfg.mach, re=cfg.re, pr=cfg.pr,
                       mu=cfg.mu, split=cfg.split, length=cfg.length,
                       offset=0.5 if (cfg.cell_centered or cfg.symmetric) else 0.0,
                       symmetric=cfg.symmetric)


def offsets(cfg: tgv.Config):
    if cfg.encoding == "offset":
        return 1.0, 1.0 / (cfg.gamma * (cfg.gamma - 1.0) * cfg.mach ** 2)
    return 0.0, 0.0


def encode(cfg: tgv.Config, q64: torch.Tensor, device="cuda") -> torch.Tensor:
    """FP64 CPU state -> device state in the storage type (offset-encoded if asked)."""
    r0, e0 = offsets(cfg)
    q = q64.clone()
    q[0] -= r0
    q[4] -= e0
    return q.to(device=device, dtype=cfg.q_dtype).contiguous()


def decode(cfg: tgv.Config, q: torch.Tensor) -> torch.Tensor:
    """Device state -> FP64 CPU state."""
    r0, e0 = offsets(cfg)
    out = q.detach().to(device="cpu", dtype=torch.float64).clone()
    out[0] += r0
    out[4] += e0
    return out


def random_state(cfg: tgv.Config, seed: int) -> torch.Tensor:
    """Smooth random (non-Taylor-Green) FP64 state around the base state."""
    flow = oracle_flow(cfg)
    rho, u, v, w, dp = (torch.from_numpy(a) for a in tgv_inputs.random_flow_fields(cfg.n, seed))
    p = 1.0 / (cfg.gamma * cfg.mach ** 2) + dp
    return oracle.conserved(flow, rho, u, v, w, p)


def rel_l2(a: torch.Tensor, b: torch.Tensor):
    """Per-field relative L2 error of a against b, fields on dim 0."""
    return [float(torch.linalg.vector_norm(a[c] - b[c]) / torch.linalg.vector_norm(b[c]))
            for c in range(a.shape[0])]


def max_rel(a: torch.Tensor, b: torch.Tensor):
    """Per-field max |a - b| / max |b|."""
    return [float((a[c] - b[c]).abs().max() / b[c].abs().max().clamp_min(1e-300))
            for c in range(a.shape[0])]


def window(q: torch.Tensor, k: int, j: int, i: int, half: int = 4) -> torch.Tensor:
    """Periodic (5, 2h, 2h, 2h) window of q with (k, j, i) at index (h, h, h)."""
    n = q.shape[-1]
    idx = lambda c: (torch.arange(c - half, c + half) % n)
    w = q[:, idx(k)][:, :, idx(j)][:, :, :, idx(i)]
    return w.contiguous()


def window_flow(cfg: tgv.Config, half: int = 4) -> oracle.Flow:
    """Oracle flow on a 2*half window with the big grid's spacing."""
    h = cfg.length / cfg.n
    return oracle_flow(cfg).with_(n=2 * half, length=2 * half * h)
