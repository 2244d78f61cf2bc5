"""FP64 CPU oracle of the Taylor-Green-vortex hot path (TEST INFRASTRUCTURE ONLY).

This module is the slow, plain reference that the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path (``paper_2505_20911_b300``) never
imports it and shares no code with it.

What it computes (arXiv 2505.20911):
  * the conservative state Q = (rho, rho*u, rho*v, rho*w, rho*E), E = e + |u|^2/2
    (Sec. 3.1);
  * the residual R(Q) = dQ/dt of the compressible Navier-Stokes equations,
    discretised with explicit 4th-order central differences for both the
    convective and the diffusive parts (Sec. 2.3.1), with the quadratic
    Blaisdell split of the convective terms d(rho u_j phi)/dx_j,
    phi in (1, u_i, E) (Sec. 2.3.1, Eq. 1 and the sentence after Eq. 2);
  * the low-storage 3-stage Runge-Kutta update
        Qt^i = A_i Qt^(i-1) + dt R^(i-1),   Q^i = Q^(i-1) + B_i Qt^i
    (Sec. 3.1, Eqs. 3-5);
  * the Taylor-Green initial condition (Sec. 4.1, Eqs. 6-10);
  * the volume-averaged kinetic energy K and the solenoidal dissipation
    eps^S (Sec. 4.1, Eqs. 11-12);
  * the gradient of the final volume-averaged kinetic energy with respect to
    the initial momentum (the discrete adjoint), by reverse-mode automatic
    differentiation of this very code (torch.autograd as the library step).

Readings where the paper defers to other papers (each is restated where it is
used):
  R1  RK coefficients: Williamson's 3-stage 2N scheme,
      A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15).
  R2  Nondimensional equations: p = (gamma-1)(rho E - rho|u|^2/2),
      T = gamma M^2 p / rho; viscous stress
      tau_ij = (mu/Re)(du_i/dx_j + du_j/dx_i - 2/3 delta_ij du_k/dx_k);
      heat flux q_j = -kappa dT/dx_j, kappa = mu / ((gamma-1) M^2 Pr Re).
  R3  Blaisdell split: C_phi = 1/2 sum_j [ D_j(rho u_j phi) + u_j D_j(rho phi)
      + rho phi D_j u_j ]; pressure terms in divergence form.  The plain
      divergence form C_phi = sum_j D_j(rho u_j phi) is kept as a foil, the
      Feiereisen quadratic split that Sec. 2.3.1 prints as its example,
        C_phi = sum_j [ 1/2 D_j(rho u_j phi) + 1/2 (phi D_j(rho u_j)
                + rho u_j D_j phi) ],
      as a second quadratic form of the study, and
      the cubic Kennedy-Gruber-Pirozzoli split of the robustness study
      (Sec. 4.2) as an alternative:
        C_phi = 1/4 sum_j [ D_j(rho u_j phi) + rho D_j(u_j phi) + u_j D_j(rho phi)
                + phi D_j(rho u_j) + rho u_j D_j phi + rho phi D_j u_j
                + u_j phi D_j rho ].
  R14 KEEP (kinetic energy and entropy preserving) split of the same study,
      which the paper cites without printing it.  Reading: the second-order
      two-point fluxes of Kuya, Totani and Kawai (2018),
        mass rho_bar u_bar,  momentum rho_bar u_bar (u_i)_bar + p_bar,
        energy rho_bar u_bar e_bar + rho_bar u_bar (u_i u_i)~/2 + (p u)~,
      (bar: mean of the two points; (a b)~ = (a_l b_r + a_r b_l)/2), carried
      to the 4th-order stencil by the two-point-flux form of central
      differences (a flux difference with weights 2 a_l over the point pairs
      l apart).  The equivalent split form, which this code evaluates: mass
      and momentum as the KGP split above; energy as the KGP split of the
      internal energy (phi = e, rho phi = p/(gamma-1)) plus
        1/4 sum_j sum_c [ rho u_j v_c D_j v_c + v_c D_j(rho u_j v_c)
                          + rho v_c D_j(u_j v_c) + u_j v_c D_j(rho v_c) ]
      for the kinetic energy, and the pressure work as
        sum_j [ u_j D_j p + p D_j u_j ].
  R4  Viscous terms, all in conservative (telescoping) form so that mass,
      momentum and total energy are conserved to round-off on the periodic box:
        momentum i: (mu/Re)[ sum_j D2_j u_i + 1/3 D2_i u_i + 1/3 D_i s_i ],
                    s_i = sum_{k != i} D_k u_k;
        heat:       kappa sum_j D2_j T;
        viscous work d(u_i tau_ij)/dx_j, rewritten exactly (product rule) as
          (mu/Re)[ sum_j D2_j(|u|^2/2) + 1/3 sum_j D2_j(u_j^2/2)
                   + 2 sum_{i<j} D_i D_j (u_i u_j) - 5/3 sum_j D_j(u_j s_j) ].
      D is the 5-point first derivative, D2 the 5-point second derivative,
      and a mixed second derivative is D_i applied after D_j.
  R5  Constant viscosity mu (1 by default, 0 for the inviscid limit), Pr = 0.71.
  R8  eps^S is normalised as a volume average, like K: eps^S = <omega.omega>/Re.
  R13 The symmetric box of Sec. 4.1 (TGSym, [0, L]^3 with symmetry planes on
      every face): cell-centred points x_i = (i + 1/2) h, h = L/N, ghosts by
      mirroring about the faces, the velocity component normal to a face odd
      and everything else even.  This is exactly the restriction to the first
      octant of the periodic problem on [0, 2L)^3 with 2N cell-centred points
      whose state is the mirror extension, and that is how it is computed here.

Array layout: a field is a float64 tensor of shape (N, N, N) indexed
[z, y, x] (x fastest, matching the device layout idx = (k*N + j)*N + i); the
state is (5, N, N, N).  Grid points x_i = i*h, h = L/N, periodic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import torch

F64 = torch.float64

# Reading R1: Williamson (1980) low-storage 3-stage, 3rd-order coefficients for
# the 2N form of Sec. 3.1, Eqs. 3-4.
RK_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)

# Field tensor dimension of each coordinate direction (x is the fastest index).
_DIM = {0: 2, 1: 1, 2: 0}


@dataclass(frozen=True)
class Flow:
    """Physical and numerical parameters of one TGV problem (Sec. 4.1)."""

    n: int
    gamma: float = 1.4
    mach: float = 0.1
    re: float = 1600.0
    pr: float = 0.71
    mu: float = 1.0
    split: str = "blaisdell"  # "divergence" (the foil), "feiereisen", "kgp" or "keep" (cubic)
    length: float = 2.0 * math.pi
    offset: float = 0.0       # grid points at (i + offset) h; 0.5 = cell-centred
    symmetric: bool = False   # symmetry planes on every face (reading R13)

    @property
    def h(self) -> float:
        return self.length / self.n

    @property
    def kappa(self) -> float:
        """Heat-conduction coefficient mu / ((gamma-1) M^2 Pr Re) (reading R2)."""
        return self.mu / ((self.gamma - 1.0) * self.mach ** 2 * self.pr * self.re)

    def with_(self, **kw) -> "Flow":
        return replace(self, **kw)


# ---------------------------------------------------------------------------
# Stencils: explicit 4th-order central differences (Sec. 2.3.1), periodic.
# ---------------------------------------------------------------------------
def shift(f: torch.Tensor, axis: int, s: int) -> torch.Tensor:
    """g[..., i, ...] = f[..., i + s, ...] along coordinate `axis` (periodic)."""
    return torch.roll(f, shifts=-s, dims=f.dim() - 3 + _DIM[axis])


def d1(f: torch.Tensor, axis: int, h: float) -> torch.Tensor:
    """4th-order central first derivative: (-f[i+2] + 8f[i+1] - 8f[i-1] + f[i-2]) / 12h."""
    return (-shift(f, axis, 2) + 8.0 * shift(f, axis, 1)
            - 8.0 * shift(f, axis, -1) + shift(f, axis, -2)) / (12.0 * h)


def d2(f: torch.Tensor, axis: int, h: float) -> torch.Tensor:
    """4th-order central second derivative:
    (-f[i+2] + 16f[i+1] - 30f[i] + 16f[i-1] - f[i-2]) / 12h^2."""
    return (-shift(f, axis, 2) + 16.0 * shift(f, axis, 1) - 30.0 * f
            + 16.0 * shift(f, axis, -1) - shift(f, axis, -2)) / (12.0 * h * h)


def grid(n: int, length: float = 2.0 * math.pi, offset: float = 0.0):
    """Coordinates (x, y, z) of the N^3 grid points (i + offset) L/N, each (N, N, N)."""
    c = (torch.arange(n, dtype=F64) + offset) * (length / n)
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    return x, y, z


# ---------------------------------------------------------------------------
# State <-> primitives (Sec. 3.1 and reading R2)
# ---------------------------------------------------------------------------
def conserved(flow: Flow, rho, u, v, w, p) -> torch.Tensor:
    """Q = (rho, rho u, rho v, rho w, rho E), rho E = p/(gamma-1) + rho|u|^2/2."""
    rhoE = p / (flow.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, rhoE])


def primitives(flow: Flow, q: torch.Tensor):
    """(rho, u, v, w, p, T) from Q; T = gamma M^2 p / rho (reading R2)."""
    rho = q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    p = (flow.gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w))
    T = flow.gamma * flow.mach ** 2 * p / rho
    return rho, u, v, w, p, T


def initial_condition(flow: Flow) -> torch.Tensor:
    """Taylor-Green initial field, Sec. 4.1, Eqs. 6-10:
    u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = 1/(gamma M^2) + (cos 2x + cos 2y)(2 + cos 2z)/16, rho = gamma M^2 p."""
    x, y, z = grid(flow.n, flow.length, 0.5 if flow.symmetric else flow.offset)
    u = torch.sin(x) * torch.cos(y) * torch.cos(z)
    v = -torch.cos(x) * torch.sin(y) * torch.cos(z)
    w = torch.zeros_like(u)
    p = 1.0 / (flow.gamma * flow.mach ** 2) + (torch.cos(2 * x) + torch.cos(2 * y)) * (
        2.0 + torch.cos(2 * z)) / 16.0
    rho = flow.gamma * flow.mach ** 2 * p
    return conserved(flow, rho, u, v, w, p)


# ---------------------------------------------------------------------------
# The residual R(Q) (Sec. 3.1), one function per group of terms.
# ---------------------------------------------------------------------------
def convective(flow: Flow, q: torch.Tensor) -> torch.Tensor:
    """C_phi for phi = (1, u, v, w, E), i.e. the discretised d(rho u_j phi)/dx_j
    (Sec. 2.3.1, Eq. 1).  Blaisdell split (reading R3):
        C_phi = 1/2 sum_j [ D_j(u_j (rho phi)) + u_j D_j(rho phi) + (rho phi) D_j u_j ],
    using rho u_j phi = u_j (rho phi); (rho phi) are the components of Q.
    Divergence form: C_phi = sum_j D_j(u_j (rho phi)).  Feiereisen (Sec. 2.3.1):
    1/2 D_j(rho u_j phi) + 1/2 (phi D_j(rho u_j) + rho u_j D_j phi).  KGP cubic form: the
    seven-term quarter average of reading R3.  KEEP (reading R14): KGP for
    phi = 1 and u_i; for the energy, KGP of the internal energy plus the
    kinetic-energy split (its pressure work is in ``pressure_terms``)."""
    h = flow.h
    rho = q[0]
    vel = (q[1] / rho, q[2] / rho, q[3] / rho)
    out = []
    for c in range(5):
        f = q[c]  # rho * phi
        if flow.split == "keep" and c == 4:
            f = primitives(flow, q)[4] / (flow.gamma - 1.0)  # rho e
        phi = f / rho
        acc = torch.zeros_like(f)
        for j in range(3):
            flux = d1(vel[j] * f, j, h)
            if flow.split == "divergence":
                acc = acc + flux
            elif flow.split == "blaisdell":
                acc = acc + 0.5 * (flux + vel[j] * d1(f, j, h) + f * d1(vel[j], j, h))
            elif flow.split == "feiereisen":
                m_j = q[1 + j]  # rho u_j
                acc = acc + 0.5 * flux + 0.5 * (phi * d1(m_j, j, h) + m_j * d1(phi, j, h))
            elif flow.split in ("kgp", "keep"):
                m_j = q[1 + j]  # rho u_j
                acc = acc + 0.25 * (flux + rho * d1(vel[j] * phi, j, h) + vel[j] * d1(f, j, h)
                                    + phi * d1(m_j, j, h) + m_j * d1(phi, j, h)
                                    + f * d1(vel[j], j, h) + vel[j] * phi * d1(rho, j, h))
                if flow.split == "keep" and c == 4:
                    for cc in range(3):  # kinetic energy: v_c = velocity component cc
                        v = vel[cc]
                        acc = acc + 0.25 * (m_j * v * d1(v, j, h) + v * d1(m_j * v, j, h)
                                            + rho * v * d1(vel[j] * v, j, h)
                                            + vel[j] * v * d1(rho * v, j, h))
            else:
                raise ValueError(f"unknown split form {flow.split!r}")
        out.append(acc)
    return torch.stack(out)


def pressure_terms(flow: Flow, q: torch.Tensor) -> torch.Tensor:
    """Pressure gradient (momentum) and pressure work (energy), divergence form:
    (0, D_x p, D_y p, D_z p, sum_j D_j(p u_j)); with KEEP (reading R14) the
    work is split as sum_j (u_j D_j p + p D_j u_j)."""
    h = flow.h
    rho, u, v, w, p, _ = primitives(flow, q)
    vel = (u, v, w)
    zero = torch.zeros_like(rho)
    if flow.split == "keep":
        work = sum(vel[j] * d1(p, j, h) + p * d1(vel[j], j, h) for j in range(3))
    else:
        work = sum(d1(p * vel[j], j, h) for j in range(3))
    return torch.stack([zero, d1(p, 0, h), d1(p, 1, h), d1(p, 2, h), work])


def viscous_terms(flow: Flow, q: torch.Tensor) -> torch.Tensor:
    """Divergence of the viscous stress and of the heat flux (reading R4):
    (0, d tau_xj/dx_j, d tau_yj/dx_j, d tau_zj/dx_j,
     d(u_i tau_ij)/dx_j - d q_j/dx_j)."""
    h = flow.h
    rho, u, v, w, p, T = primitives(flow, q)
    vel = (u, v, w)
    nu = flow.mu / flow.re
    # Diagonal velocity gradients D_k u_k and s_i = sum_{k != i} D_k u_k.
    diag = [d1(vel[k], k, h) for k in range(3)]
    s = [sum(diag[k] for k in range(3) if k != i) for i in range(3)]
    mom = []
    for i in range(3):
        lap = sum(d2(vel[i], j, h) for j in range(3))
        mom.append(nu * (lap + d2(vel[i], i, h) / 3.0 + d1(s[i], i, h) / 3.0))
    ke = 0.5 * (u * u + v * v + w * w)
    work = torch.zeros_like(rho)
    for j in range(3):
        work = work + d2(ke, j, h) + d2(0.5 * vel[j] * vel[j], j, h) / 3.0
        work = work - (5.0 / 3.0) * d1(vel[j] * s[j], j, h)
    for i in range(3):
        for j in range(i + 1, 3):
            work = work + 2.0 * d1(d1(vel[i] * vel[j], j, h), i, h)
    heat = flow.kappa * sum(d2(T, j, h) for j in range(3))
    zero = torch.zeros_like(rho)
    return torch.stack([zero, mom[0], mom[1], mom[2], nu * work + heat])


def mirror_extend(q: torch.Tensor) -> torch.Tensor:
    """(5, N, N, N) state of the symmetric box -> (5, 2N, 2N, 2N) periodic state:
    along each axis the second half is the mirror image of the first, with the
    momentum component normal to that axis negated (reading R13)."""
    out = q
    for axis, dim in ((0, 3), (1, 2), (2, 1)):
        m = torch.flip(out, dims=[dim]).clone()
        m[1 + axis] = -m[1 + axis]
        out = torch.cat([out, m], dim=dim)
    return out


def _periodic_twin(flow: Flow) -> Flow:
    return flow.with_(n=2 * flow.n, length=2 * flow.length, offset=0.5, symmetric=False)


def residual(flow: Flow, q: torch.Tensor) -> torch.Tensor:
    """R(Q) = dQ/dt = -C - (pressure terms) + (viscous and heat terms)."""
    if flow.symmetric:
        n = flow.n
        return residual(_periodic_twin(flow), mirror_extend(q))[:, :n, :n, :n]
    r = -convective(flow, q) - pressure_terms(flow, q)
    if flow.mu != 0.0:
        r = r + viscous_terms(flow, q)
    return r


# ---------------------------------------------------------------------------
# Low-storage RK3 (Sec. 3.1, Eqs. 3-5)
# ---------------------------------------------------------------------------
def rk_substep(flow: Flow, q, qt, i: int, dt: float, rhs=None):
    """One substep i (0-based): Qt <- A_i Qt + dt R(Q); Q <- Q + B_i Qt."""
    r = (rhs or (lambda x: residual(flow, x)))(q)
    qt = RK_A[i] * qt + dt * r
    return q + RK_B[i] * qt, qt


def rk3_step(flow: Flow, q, dt: float, rhs=None):
    """Q^n -> Q^{n+1} = Q^m after m = 3 substeps; Qt starts at zero (A_1 = 0)."""
    qt = torch.zeros_like(q)
    for i in range(3):
        q, qt = rk_substep(flow, q, qt, i, dt, rhs)
    return q


def run(flow: Flow, q, dt: float, nsteps: int, log_every: int = 0):
    """Advance nsteps; optionally return diagnostics every log_every steps."""
    log = []
    for n in range(nsteps):
        if log_every and n % log_every == 0:
            log.append((n, diagnostics(flow, q)))
        q = rk3_step(flow, q, dt)
    if log_every:
        log.append((nsteps, diagnostics(flow, q)))
        return q, log
    return q


# ---------------------------------------------------------------------------
# Diagnostics (Sec. 4.1, Eqs. 11-12; reading R8)
# ---------------------------------------------------------------------------
DIAG_NAMES = ("K", "K_rho", "enstrophy", "eps_S", "rho", "rho_u", "rho_v",
              "rho_w", "rho_E", "nonfinite")


def vorticity(flow: Flow, q):
    if flow.symmetric:
        n = flow.n
        return tuple(c[:n, :n, :n] for c in vorticity(_periodic_twin(flow), mirror_extend(q)))
    h = flow.h
    _, u, v, w, _, _ = primitives(flow, q)
    wx = d1(w, 1, h) - d1(v, 2, h)
    wy = d1(u, 2, h) - d1(w, 0, h)
    wz = d1(v, 0, h) - d1(u, 1, h)
    return wx, wy, wz


def kinetic_energy(flow: Flow, q) -> torch.Tensor:
    """K = (1/V) int u_i u_i / 2 dV, the grid mean on a uniform periodic grid."""
    _, u, v, w, _, _ = primitives(flow, q)
    return (0.5 * (u * u + v * v + w * w)).mean()


def diagnostics(flow: Flow, q) -> dict:
    """K, <rho|u|^2/2>, <omega.omega>, eps^S = <omega.omega>/Re, means of Q,
    and the count of non-finite points."""
    rho, u, v, w, _, _ = primitives(flow, q)
    wx, wy, wz = vorticity(flow, q)
    ens = (wx * wx + wy * wy + wz * wz).mean()
    out = {
        "K": float(kinetic_energy(flow, q)),
        "K_rho": float((0.5 * rho * (u * u + v * v + w * w)).mean()),
        "enstrophy": float(ens),
        "eps_S": float(ens / flow.re),
        "rho": float(q[0].mean()),
        "rho_u": float(q[1].mean()),
        "rho_v": float(q[2].mean()),
        "rho_w": float(q[3].mean()),
        "rho_E": float(q[4].mean()),
        "nonfinite": float((~torch.isfinite(q)).any(dim=0).sum()),
    }
    return out


# ---------------------------------------------------------------------------
# Discrete adjoint: gradient of J = K(Q_N) w.r.t. the initial momentum.
# ---------------------------------------------------------------------------
def final_ke(flow: Flow, q0, dt: float, nsteps: int):
    """J = K(Q_nsteps) for the run started from q0."""
    return kinetic_energy(flow, run(flow, q0, dt, nsteps))


def grad_final_ke(flow: Flow, q0, dt: float, nsteps: int, ckpt_every: int = 1):
    """(J, dJ/d(rho u_0, rho v_0, rho w_0)) with rho_0 and (rho E)_0 held fixed.

    Reverse-mode differentiation of the discrete map Q_0 -> Q_N, one time step
    at a time: Q_n is recomputed from the last stored checkpoint, the step is
    re-run under autograd, and the cotangent is pulled back through it.
    """
    with torch.no_grad():
        ckpts = {}
        q = q0.clone()
        for n in range(nsteps):
            if n % ckpt_every == 0:
                ckpts[n] = q.clone()
            q = rk3_step(flow, q, dt)
    qn = q.clone().requires_grad_(True)
    J = kinetic_energy(flow, qn)
    (lam,) = torch.autograd.grad(J, qn)
    for n in reversed(range(nsteps)):
        base = (n // ckpt_every) * ckpt_every
        with torch.no_grad():
            q = ckpts[base].clone()
            for m in range(base, n):
                q = rk3_step(flow, q, dt)
        q = q.requires_grad_(True)
        out = rk3_step(flow, q, dt)
        (lam,) = torch.autograd.grad(out, q, grad_outputs=lam)
    return float(J), lam[1:4].clone()


def rhs_vjp(flow: Flow, q, lam):
    """(dR/dQ)^T lam at state q."""
    q = q.clone().requires_grad_(True)
    r = residual(flow, q)
    (g,) = torch.autograd.grad(r, q, grad_outputs=lam)
    return g


def rhs_jvp(flow: Flow, q, v):
    """(dR/dQ) v at state q (forward mode)."""
    _, jv = torch.func.jvp(lambda x: residual(flow, x), (q,), (v,))
    return jv
