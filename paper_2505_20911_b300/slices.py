"""Headless output of the flow field: planes of the state as .npy arrays.

The paper shows the flow as contour images of rho E on planes through the box
(Sec. 4, the Taylor-Green snapshots).  This library renders nothing; it writes
the decoded plane arrays that a plotting tool reads.  A plane is taken from the
state Q (device or host tensor, the library's [5][N][N][N] layout with x
fastest, so q[c, z, y, x]), copied to the host, widened to FP64 and, with the
offset encoding, given back the uniform base state that the stored rho and
rho E omit.
"""
from __future__ import annotations

import os

import numpy as np
import torch

FIELDS = ("rho", "rho_u", "rho_v", "rho_w", "rho_E")
_AXES = {"z": 1, "y": 2, "x": 3}


def encoding_offsets(cfg) -> tuple[float, float]:
    """(rho_0, (rho E)_0) that the offset encoding subtracts from the stored
    rho and rho E (the uniform base state rho = 1, rho E = 1/(gamma (gamma-1)
    M^2)); zeros for the plain encoding."""
    if cfg.encoding == "offset":
        return 1.0, 1.0 / (cfg.gamma * (cfg.gamma - 1.0) * cfg.mach * cfg.mach)
    return 0.0, 0.0


def plane(cfg, q: torch.Tensor, axis: str = "z", index: int | None = None,
          fields=FIELDS) -> dict[str, np.ndarray]:
    """The decoded conserved fields on the plane `axis` = `index` (default: the
    mid-plane N/2) as FP64 arrays of shape (N, N), keyed by field name.  For
    axis "z" the array is indexed [y, x], for "y" [z, x], for "x" [z, y]."""
    n = cfg.n
    if tuple(q.shape) != (5, n, n, n):
        raise ValueError(f"q must have shape (5, {n}, {n}, {n}), got {tuple(q.shape)}")
    if axis not in _AXES:
        raise ValueError(f"axis must be one of {sorted(_AXES)}")
    idx = n // 2 if index is None else int(index)
    if not 0 <= idx < n:
        raise ValueError(f"index {idx} outside 0..{n - 1}")
    unknown = [f for f in fields if f not in FIELDS]
    if unknown:
        raise ValueError(f"unknown fields {unknown}; choose from {FIELDS}")
    sl = q.detach().select(_AXES[axis], idx).to("cpu", torch.float64).numpy()
    rho0, rhoE0 = encoding_offsets(cfg)
    out = {}
    for f in fields:
        c = FIELDS.index(f)
        a = sl[c].copy()
        if c == 0:
            a += rho0
        elif c == 4:
            a += rhoE0
        out[f] = a
    return out


def save_midplane_slices(directory: str, cfg, q: torch.Tensor, axes=("z",), fields=("rho_E",),
                         step: int | None = None) -> list[str]:
    """Write the mid-plane of each field on each axis as
    `<directory>/<field>_<axis><index>[_s<step>].npy`; returns the paths."""
    os.makedirs(directory, exist_ok=True)
    paths = []
    for ax in axes:
        arrays = plane(cfg, q, ax, None, fields)
        for f, a in arrays.items():
            tag = f"_s{step}" if step is not None else ""
            p = os.path.join(directory, f"{f}_{ax}{cfg.n // 2}{tag}.npy")
            np.save(p, a)
            paths.append(p)
    return paths
