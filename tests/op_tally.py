"""Floating-point operation tally of one Runge-Kutta stage per grid point,
counted from the FP64 oracle's formulas (test infrastructure; it runs the
oracle).

The oracle evaluates the residual of Sec. 3.1 (the split convective terms of
Sec. 2.3.1, the pressure terms, the viscous stress and heat flux) and the
2N update of Eqs. 3-4 with plain elementwise tensor arithmetic.  This script
runs one stage on a small periodic grid under a dispatch mode that sees every
arithmetic operator and counts, per grid point:

  add/sub, mul, div (each 1 flop), neg (0 flops: a sign change the hardware
  folds into the next operation), one entry per distinct result.

"Distinct" is what makes the count algorithmic rather than a count of the
oracle's own redundancy: the oracle recomputes the primitives in each group
of terms and some derivatives twice (e.g. D2_i u_i in the Laplacian and in
the 1/3 D2_i u_i term).  An operation whose operator and operand values equal
those of an operation already counted is counted once, as a kernel that
computes each quantity once would.  Data movement (the periodic shifts of
the stencils, stacking, copies) costs nothing.

Running it as a script prints the tally per term group and per split form
and writes the Markdown summary that bench.py reads (profiles/op_tally.md):

    python tests/op_tally.py
"""
from __future__ import annotations

import hashlib
import os
import sys

import torch
from torch.utils._python_dispatch import TorchDispatchMode, _disable_current_modes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import tgv_inputs  # noqa: E402

aten = torch.ops.aten
FLOP_OPS = {
    aten.add: ("add", 1), aten.sub: ("add", 1), aten.rsub: ("add", 1),
    aten.mul: ("mul", 1), aten.div: ("div", 1), aten.neg: ("neg", 0),
}


def _fingerprint(x):
    if isinstance(x, torch.Tensor):
        with _disable_current_modes():
            b = x.detach().contiguous().cpu().numpy().tobytes()
        return ("T", tuple(x.shape), str(x.dtype), hashlib.blake2b(b, digest_size=16).hexdigest())
    return ("S", repr(x))


class OpCounter(TorchDispatchMode):
    """Counts elementwise arithmetic results (per element), each distinct
    (operator, operand values) once."""

    def __init__(self):
        super().__init__()
        self.seen = set()
        self.counts = {"add": 0, "mul": 0, "div": 0, "neg": 0}
        self.flops = 0
        self.repeats = 0

    def __torch_dispatch__(self, func, types, args=(), kwargs=None):
        out = func(*args, **(kwargs or {}))
        kind = FLOP_OPS.get(func.overloadpacket)
        if kind is not None and isinstance(out, torch.Tensor):
            ops = list(args)
            if func.overloadpacket in (aten.add, aten.mul):   # commutative
                ops = sorted(ops, key=lambda a: repr(_fingerprint(a)))
            key = (kind[0], tuple(_fingerprint(a) for a in ops),
                   tuple(sorted((k, repr(v)) for k, v in (kwargs or {}).items())))
            if key in self.seen:
                self.repeats += out.numel()
            else:
                self.seen.add(key)
                self.counts[kind[0]] += out.numel()
                self.flops += kind[1] * out.numel()
        return out


def tally(split: str = "blaisdell", n: int = 8, mu: float = 1.0, seed: int = 3):
    """Per-point counts of one RK stage (residual + the 2N update), by group.

    A random smooth state (no symmetry, so no two distinct quantities share
    their values by accident) on an n^3 periodic grid.  Returns
    {group: {"add", "mul", "div", "neg", "flops"}} per grid point."""
    flow = oracle.Flow(n=n, mu=mu, split=split)
    rho, u, v, w, dp = (torch.from_numpy(a) for a in tgv_inputs.random_flow_fields(n, seed))
    p = 1.0 / (flow.gamma * flow.mach ** 2) + dp
    q = oracle.conserved(flow, rho, u, v, w, p)
    qt = torch.randn(q.shape, dtype=q.dtype, generator=torch.Generator().manual_seed(seed))
    pts = n ** 3
    groups = {}
    c = OpCounter()  # one counter across groups: a quantity shared by two groups counts once
    with c:
        steps = [
            ("convective", lambda: oracle.convective(flow, q)),
            ("pressure", lambda: oracle.pressure_terms(flow, q)),
            ("viscous+heat", lambda: oracle.viscous_terms(flow, q) if mu != 0.0 else None),
            ("assembly", lambda: oracle.residual(flow, q)),
            ("rk update", lambda: oracle.rk_substep(flow, q, qt, 1, 1e-3)),
        ]
        prev = dict(c.counts, flops=0)
        for name, fn in steps:
            fn()
            now = dict(c.counts, flops=c.flops)
            groups[name] = {k: (now[k] - prev.get(k, 0)) / pts for k in now}
            prev = now
    groups["total"] = {k: sum(g[k] for g in groups.values()) for k in groups["convective"]}
    groups["_repeats"] = c.repeats / pts
    return groups


def write_summary(path: str) -> dict:
    splits = ("blaisdell", "divergence", "feiereisen", "kgp", "keep")
    res = {s: tally(s) for s in splits}
    lines = [
        "# Floating-point operations per grid point and RK stage, counted from the oracle",
        "",
        "Command: `python tests/op_tally.py` (runs the FP64 oracle on a random 8^3 state",
        "under an operator-counting dispatch mode; each distinct (operator, operand values)",
        "counted once; add/sub, mul, div = 1 flop, neg = 0).",
        "",
        "| split | group | add/sub | mul | div | flops |",
        "|---|---|---:|---:|---:|---:|",
    ]
    for s in splits:
        for g in ("convective", "pressure", "viscous+heat", "assembly", "rk update", "total"):
            t = res[s][g]
            lines.append(f"| {s} | {g} | {t['add']:.0f} | {t['mul']:.0f} | {t['div']:.0f} | "
                         f"{t['flops']:.0f} |")
    lines += ["", "Machine-read by bench.py:", ""]
    for s in splits:
        lines.append(f"- flops_per_point_stage_{s}: `{res[s]['total']['flops']:.0f}`")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return res


if __name__ == "__main__":
    out = write_summary(os.path.join(ROOT, "profiles", "op_tally.md"))
    for s, g in out.items():
        print(s, {k: round(v["flops"], 1) for k, v in g.items() if isinstance(v, dict)},
              "repeats skipped:", round(g["_repeats"], 1))
