"""Pins of the oracle's residual R(Q) (CPU only).

* Convergence at 4th order (Sec. 2.3.1) to the exact continuous right-hand
  side of the compressible Navier-Stokes equations, derived symbolically here
  from their textbook conservative form (not from the split or the rewritten
  viscous work the oracle uses), group by group and in total.
* Discrete conservation of mass, momentum and total energy on the periodic
  box to round-off (telescoping sums).
* The skew-symmetry identity that characterises the Blaisdell split:
  sum_x f C_f = 1/2 sum_x (D_j u_j) f^2 for every conserved component f.
* The Taylor-Green symmetries of the initial field are kept by R.
"""
import math

import numpy as np
import pytest
import sympy as sp
import torch

import oracle
import tgv_inputs

GAMMA, MACH, RE, PR = 1.4, 0.5, 20.0, 0.71


def _exact_groups():
    """Exact convective, pressure and viscous groups for a manufactured field."""
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    g, M, Re, Pr, mu = sp.Float(GAMMA), sp.Float(MACH), sp.Float(RE), sp.Float(PR), sp.Integer(1)
    rho = 1 + sp.Rational(1, 10) * sp.sin(x + 2 * y - z)
    u = sp.sin(x) * sp.cos(y) * sp.cos(z) + sp.Rational(3, 10) * sp.sin(y + z)
    v = -sp.cos(x) * sp.sin(y) * sp.cos(z) + sp.Rational(1, 5) * sp.cos(x - z)
    w = sp.Rational(3, 10) * sp.sin(x + y) * sp.cos(2 * z)
    p = 1 / (g * M ** 2) + sp.Rational(1, 10) * sp.cos(2 * x - y) * sp.sin(z)
    vel = (u, v, w)
    rhoE = p / (g - 1) + rho * (u ** 2 + v ** 2 + w ** 2) / 2
    T = g * M ** 2 * p / rho
    kappa = mu / ((g - 1) * M ** 2 * Pr * Re)
    div = sum(sp.diff(vel[k], X[k]) for k in range(3))
    tau = [[mu / Re * (sp.diff(vel[i], X[j]) + sp.diff(vel[j], X[i])
                       - (sp.Rational(2, 3) * div if i == j else 0))
            for j in range(3)] for i in range(3)]
    phis = (sp.Integer(1), u, v, w, rhoE / rho)
    conv = [sum(sp.diff(rho * vel[j] * phi, X[j]) for j in range(3)) for phi in phis]
    pres = [sp.Integer(0)] + [sp.diff(p, X[i]) for i in range(3)] + \
           [sum(sp.diff(p * vel[j], X[j]) for j in range(3))]
    visc = [sp.Integer(0)] + [sum(sp.diff(tau[i][j], X[j]) for j in range(3)) for i in range(3)]
    visc.append(sum(sp.diff(sum(vel[i] * tau[i][j] for i in range(3)), X[j]) for j in range(3))
                + sum(sp.diff(kappa * sp.diff(T, X[j]), X[j]) for j in range(3)))
    prim = (rho, u, v, w, p)
    f = lambda exprs: [sp.lambdify((x, y, z), e, "numpy") for e in exprs]
    return f(prim), f(conv), f(pres), f(visc)


@pytest.fixture(scope="module")
def exact():
    return _exact_groups()


def _eval(fns, n):
    x, y, z = oracle.grid(n)
    out = []
    for fn in fns:
        val = fn(x.numpy(), y.numpy(), z.numpy())
        out.append(torch.as_tensor(np.broadcast_to(val, x.shape).copy(), dtype=torch.float64))
    return out


def _errors(exact, group, n):
    prim_fns, conv_fns, pres_fns, visc_fns = exact
    flow = oracle.Flow(n=n, gamma=GAMMA, mach=MACH, re=RE, pr=PR)
    rho, u, v, w, p = _eval(prim_fns, n)
    q = oracle.conserved(flow, rho, u, v, w, p)
    if group == "convective":
        disc, ref = oracle.convective(flow, q), torch.stack(_eval(conv_fns, n))
    elif group == "pressure":
        disc, ref = oracle.pressure_terms(flow, q), torch.stack(_eval(pres_fns, n))
    elif group == "viscous":
        disc, ref = oracle.viscous_terms(flow, q), torch.stack(_eval(visc_fns, n))
    else:
        disc = oracle.residual(flow, q)
        ref = -torch.stack(_eval(conv_fns, n)) - torch.stack(_eval(pres_fns, n)) \
            + torch.stack(_eval(visc_fns, n))
    return [(float((disc[c] - ref[c]).abs().max()), float(ref[c].abs().max())) for c in range(5)]


@pytest.mark.parametrize("group", ["convective", "pressure", "viscous", "total"])
def test_residual_converges_at_fourth_order(exact, group):
    e32 = _errors(exact, group, 32)
    e64 = _errors(exact, group, 64)
    for c in range(5):
        (a, scale), (b, _) = e32[c], e64[c]
        if scale < 1e-12:  # an identically zero component (mass in the viscous group)
            assert a < 1e-12 and b < 1e-12
            continue
        assert b < 1e-3 * scale, (group, c, b, scale)
        assert a / b > 13.0, (group, c, a, b)


@pytest.mark.parametrize("split", ["divergence", "feiereisen", "kgp", "keep"])
def test_other_split_forms_converge_to_same_rhs(exact, split):
    prim_fns, conv_fns, _, _ = exact
    errs = []
    for n in (32, 64):
        flow = oracle.Flow(n=n, gamma=GAMMA, mach=MACH, re=RE, pr=PR, split=split)
        q = oracle.conserved(flow, *_eval(prim_fns, n))
        ref = torch.stack(_eval(conv_fns, n))
        errs.append(float((oracle.convective(flow, q) - ref).abs().max()))
    assert errs[0] / errs[1] > 13.0, errs


def _random_state(n, seed, mach=0.3):
    flow = oracle.Flow(n=n, mach=mach, re=50.0)
    rho, u, v, w, dp = (torch.from_numpy(a) for a in tgv_inputs.random_flow_fields(n, seed))
    p = 1.0 / (flow.gamma * mach ** 2) + dp
    return flow, oracle.conserved(flow, rho, u, v, w, p)


@pytest.mark.parametrize("split", ["blaisdell", "divergence", "feiereisen", "kgp", "keep"])
def test_discrete_conservation(split):
    flow, q = _random_state(16, 3)
    flow = flow.with_(split=split)
    r = oracle.residual(flow, q)
    for c in range(5):
        scale = float(r[c].abs().max())
        assert abs(float(r[c].sum())) / r[c].numel() < 1e-14 * max(scale, 1.0), (c, float(r[c].sum()))


def test_blaisdell_skew_identity():
    flow, q = _random_state(16, 5)
    conv = oracle.convective(flow, q)
    rho = q[0]
    div = sum(oracle.d1(q[1 + j] / rho, j, flow.h) for j in range(3))
    for c in range(5):
        lhs = float((q[c] * conv[c]).sum())
        rhs = float((0.5 * div * q[c] * q[c]).sum())
        scale = float((q[c] * q[c]).abs().sum()) * float(div.abs().max())
        assert abs(lhs - rhs) < 1e-13 * scale, (c, lhs, rhs)
    # The divergence form does not have this property.
    dflow = flow.with_(split="divergence")
    conv_d = oracle.convective(dflow, q)
    c = 1
    gap = abs(float((q[c] * conv_d[c]).sum()) - float((0.5 * div * q[c] * q[c]).sum()))
    assert gap > 1e-6 * float((q[c] * q[c]).abs().sum())


def _tgv_symmetry_ops(n):
    """Symmetries of the Taylor-Green field (Sec. 4.1, Eqs. 6-10) acting on a
    state (5, N, N, N): mirrors x -> -x, y -> -y, z -> -z with the matching
    velocity component negated, and the swap x <-> y (exchanging u and v)
    followed by a shift of pi in z."""
    mirror = lambda f, d: torch.roll(torch.flip(f, dims=[d]), 1, dims=d)

    def mir(q, axis):
        d = {0: -1, 1: -2, 2: -3}[axis]
        out = torch.stack([mirror(q[c], d) for c in range(5)])
        out[1 + axis] = -out[1 + axis]
        return out

    def swap_shift(q):
        sw = lambda f: torch.roll(f.transpose(-1, -2), n // 2, dims=-3)
        return torch.stack([sw(q[0]), sw(q[2]), sw(q[1]), sw(q[3]), sw(q[4])])

    return [lambda q: mir(q, 0), lambda q: mir(q, 1), lambda q: mir(q, 2), swap_shift]


def test_residual_keeps_tgv_symmetries():
    flow = oracle.Flow(n=16)
    q = oracle.initial_condition(flow)
    r = oracle.residual(flow, q)
    for op in _tgv_symmetry_ops(flow.n):
        assert torch.allclose(op(q), q, rtol=0, atol=1e-13 * float(q.abs().max()))
        assert torch.allclose(op(r), r, rtol=0, atol=1e-12 * float(r.abs().max()))


def test_kgp_kinetic_energy_identity():
    """The cubic KGP split makes the convective transport of kinetic energy a
    telescoping sum: sum_x [u_i C_(rho u_i) - |u|^2/2 C_rho] = 0 (a discrete
    property of the form; the Blaisdell and divergence forms do not have it)."""
    flow, q = _random_state(16, 9)
    rho = q[0]
    u = [q[1 + i] / rho for i in range(3)]
    ke = 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)

    def imbalance(split):
        conv = oracle.convective(flow.with_(split=split), q)
        s = sum(u[i] * conv[1 + i] for i in range(3)) - ke * conv[0]
        return abs(float(s.sum())) / float((u[0] * conv[1]).abs().sum())
    assert imbalance("kgp") < 1e-13, imbalance("kgp")
    assert imbalance("keep") < 1e-13, imbalance("keep")
    assert imbalance("blaisdell") > 1e-6 and imbalance("divergence") > 1e-6


def test_feiereisen_skew_part_is_zero_sum_and_linear_case():
    """Feiereisen (Sec. 2.3.1): the part 1/2 (phi D(rho u) + rho u D phi) sums
    to zero over the periodic box (D is skew), and with phi constant (the
    mass equation) the split reduces to the divergence form D(rho u_j)."""
    flow, q = _random_state(16, 13)
    conv_f = oracle.convective(flow.with_(split="feiereisen"), q)
    conv_d = oracle.convective(flow.with_(split="divergence"), q)
    assert torch.allclose(conv_f[0], conv_d[0], rtol=0, atol=1e-12 * float(conv_d[0].abs().max()))
    for c in range(1, 5):
        skew = 2.0 * (conv_f[c] - 0.5 * conv_d[c])
        assert abs(float(skew.sum())) < 1e-12 * float(skew.abs().sum()), c


def test_keep_equals_its_two_point_flux_form():
    """Reading R14 defines KEEP by two-point fluxes; the oracle evaluates an
    expanded split form.  Pin: the conservative flux difference built here
    directly from the two-point fluxes,
        delta_j F = (2/h) sum_(l=1,2) a_l [F(q_i, q_(i+l)) - F(q_(i-l), q_i)],
        a_1 = 2/3, a_2 = -1/12 (the weights of the 4th-order D),
    equals the oracle's convective plus pressure terms for all five equations."""
    flow, q = _random_state(16, 21)
    flow = flow.with_(split="keep")
    g1 = flow.gamma - 1.0
    rho = q[0]
    vel = [q[1 + i] / rho for i in range(3)]
    p = g1 * (q[4] - 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    e = p / (g1 * rho)
    dim = {0: 2, 1: 1, 2: 0}

    def flux(a, b, j):
        """Two-point KEEP fluxes in direction j between states a and b."""
        ra, rb = a[0], b[0]
        ua, ub = a[1 + j], b[1 + j]
        mass = (ra + rb) * (ua + ub) / 4.0
        mom = [mass * (a[1 + c] + b[1 + c]) / 2.0 + ((a[4] + b[4]) / 2.0 if c == j else 0.0)
               for c in range(3)]
        vv = a[1] * b[1] + a[2] * b[2] + a[3] * b[3]
        energy = mass * (a[5] + b[5]) / 2.0 + mass * vv / 2.0 + (a[4] * ub + b[4] * ua) / 2.0
        return [mass] + mom + [energy]

    prim = torch.stack([rho, vel[0], vel[1], vel[2], p, e])   # (rho, u, v, w, p, e)
    total = torch.zeros_like(q)
    for j in range(3):
        sh = lambda f, l: torch.roll(f, -l, dims=1 + dim[j])   # value at i + l
        for l, a_l in ((1, 2.0 / 3.0), (2, -1.0 / 12.0)):
            right = flux(prim, sh(prim, l), j)
            left = flux(sh(prim, -l), prim, j)
            for c in range(5):
                total[c] += 2.0 * a_l * (right[c] - left[c]) / flow.h
    split_form = oracle.convective(flow, q) + oracle.pressure_terms(flow, q)
    for c in range(5):
        scale = float(split_form[c].abs().max())
        assert float((total[c] - split_form[c]).abs().max()) < 1e-12 * scale, c
