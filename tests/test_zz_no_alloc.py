"""diagnostics_reduce_noalloc, the entry point for callers that cannot
allocate device memory (it keeps its partial sums in a fixed array inside the
library), must give what diagnostics_reduce gives with a caller workspace.

This file is named to be collected last, so a failure here comes after every
other test has run; it also passes on its own in a fresh process."""
import pytest
import torch

import paper_2505_20911_b300 as tgv
from _util import encode, random_state

pytestmark = pytest.mark.gpu


def _via_workspace(cfg, q):
    out = torch.empty(tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
    tgv.diagnostics_reduce(cfg, q, out, tgv.empty_workspace(cfg))
    return out.cpu()


def _via_noalloc(cfg, q):
    out = torch.full((tgv.TGV_DIAG_COUNT,), float("nan"), dtype=torch.float64, device="cuda")
    tgv.diagnostics_reduce_noalloc(cfg, q, out)
    return out.cpu()


def test_noalloc_diagnostics_match_workspace_version_twice_in_a_row():
    # two calls in a row on different states and sizes: the second must not
    # see anything the first left in the shared array
    cases = [(tgv.Config(n=48, mode="fp64", mach=0.3, re=50.0), 21),
             (tgv.Config(n=32, mode="fp32", mach=0.2, re=400.0), 22)]
    for cfg, seed in cases:
        q = encode(cfg, random_state(cfg, seed))
        ref = _via_workspace(cfg, q)
        got = _via_noalloc(cfg, q)
        torch.cuda.synchronize()
        for m, name in enumerate(tgv.DIAG_NAMES):
            assert abs(float(got[m]) - float(ref[m])) <= 1e-12 * abs(float(ref[m])) + 1e-15, \
                (cfg.n, name, float(got[m]), float(ref[m]))
