"""The operation tally (tests/op_tally.py) counts what the oracle's formulas
state, and the committed summary that bench.py reads is reproducible."""
import os
import re

import pytest

import op_tally

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counter_matches_a_hand_count_of_the_divergence_form():
    """Divergence form, Sec. 2.3.1: C_c = sum_j D_j(u_j f_c).  Per point: the
    15 products u_j f_c (1 mul each); 15 first derivatives as the oracle writes
    them, (-f[+2] + 8 f[+1] - 8 f[-1] + f[-2]) / (12 h): 2 mul + 3 add + 1 div
    (the leading minus is a sign change, 0 flops); 15 accumulations over
    (c, j) starting from a zero array; the velocities u_j = (rho u_j)/rho and
    phi = f/rho for c = 0 and c = 4 (u_j already counted): 5 div."""
    t = op_tally.tally("divergence", mu=0.0)
    assert t["convective"]["flops"] == 15 * 1 + 15 * 6 + 15 + 5
    assert t["convective"]["div"] == 15 + 5


def test_blaisdell_adds_the_two_skew_terms():
    """Blaisdell = divergence + per (c, j) the terms u_j D_j f_c and f_c D_j u_j,
    their sum with the flux and the factor 1/2 (2 mul, 2 add, 1 mul per (c, j)),
    the derivatives D_j f_c (15 D's, 6 flops each) and D_j u_j (3 D's); the
    divergence form's mass fluxes D_j(u_j rho) are the same numbers as
    D_j(rho u_j) (u_j rho reproduces rho u_j exactly on this state), so those
    3 D's are not new."""
    div = op_tally.tally("divergence", mu=0.0)["convective"]["flops"]
    bla = op_tally.tally("blaisdell", mu=0.0)["convective"]["flops"]
    assert bla == div + 15 * 5 + 15 * 6 + 3 * 6 - 3 * 6


@pytest.mark.parametrize("split", ["blaisdell", "kgp"])
def test_committed_summary_is_reproducible(split):
    text = open(os.path.join(ROOT, "profiles", "op_tally.md")).read()
    m = re.search(rf"flops_per_point_stage_{split}: `(\d+)`", text)
    assert m, split
    assert int(m.group(1)) == round(op_tally.tally(split)["total"]["flops"])
