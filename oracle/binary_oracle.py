"""FP64 CPU oracle of the binary-fluid free-energy lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Like ``lb_oracle``, this module is imported by
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``;
nothing on the product path imports, calls or links it, and it imports
nothing from there.  It reuses ``lb_oracle``'s velocity sets, weights,
stencils, shift, Eq. 28 body force and Eq. 27 force populations (the same
oracle package), which are pinned by their own tests.

The paper (Sec. I) says its analysis of the liquid-gas scheme applies equally
to other multiphase systems solved by the free-energy method, binary fluids
among them, but prints no equation for them.  The model below is the reading
used here; every step is the liquid-gas construction of Secs. II-VI with the
order parameter phi in place of the density wherever a gradient enters:

* B1  Free energy (symmetric binary fluid, two components of equal mass):
      psi = rho/3 ln rho + A/2 phi^2 + B/4 phi^4 + kappa/2 |grad phi|^2,
      A < 0 < B; bulk phases phi = +-phi*, phi* = sqrt(-A/B).
* B2  Chemical potential mu = A phi + B phi^3 - kappa lap(phi); bulk pressure
      p0 = rho dpsi/drho + phi dpsi/dphi - psi = rho/3 + A/2 phi^2 + 3B/4 phi^4.
* B3  Pressure tensor (Eq. 1 with rho -> phi in its gradient terms):
      P_ab = (p0 - kappa phi lap(phi) - kappa/2 |grad phi|^2) d_ab
             + kappa d_a phi d_b phi.
* B4  f^eq: Eqs. 5 and 6 with this p0, w^t_i kappa phi lap(phi) and
      w^ab_i kappa d_a phi d_b phi, and lambda = 0 (Eq. 36: c_s^2 = dp0/drho
      = 1/3 at fixed phi, so nu (1 - 3 c_s^2) vanishes).
* B5  g^eq (order parameter), the moments sum g = phi, sum g e = phi u,
      sum g e_a e_b = Gamma mu d_ab + phi u_a u_b:
      g_i = (w_i/c^2)(e_ia phi u_a + 3/(2c^2)[e_ia e_ib - c^2/3 d_ab] phi u_a u_b)
            + w^p_i Gamma mu / c^2  (i >= 1),   g_0 = phi - sum_{i>=1} g_i.
* B6  g relaxes with its own time tau_phi (mobility Gamma (tau_phi - 1/2)),
      without a force term, and streams like f.
* B7  Forcing scheme (Sec. VI): the M terms leave f^eq and act as the body
      force of Eq. 28 with M_ab = kappa d_a phi d_b phi (force stencil (E, F),
      reading R6; in 3D reading R7); F_i by Eq. 27 (reading R8); the fluid
      velocity is v = u + g/(2 rho) (Eq. 40), and g^eq takes v in place of u,
      so that the order parameter moves with the fluid: with u, which stays
      -g/(2 rho) in a resting interface, the flux phi u never vanishes, mu
      never becomes uniform and a flat interface drifts away from its
      profile (measured: 4% of phi* after 1600 steps and growing, against a
      converged 1.5% with v).
* B8  Stencils: the gradient and Laplacian of phi are Eq. 10 / Eq. 11
      (Eq. 29 in 3D) at the paper's optimum coefficients.

Both lattices: D2Q9 with the weights of Sec. VIII, D3Q19 with those of Eq. 31
(readings R4, R5), the forcing scheme in 3D by reading R7.

Parity status: pinned by ``tests/test_binary_oracle.py`` (reduction to the
textbook D2Q9 equilibrium, the moments of f^eq and g^eq against the closed
forms B3 / B5, exact conservation of mass, order parameter and momentum, the
stationary flat interface phi* tanh(x / w), w = sqrt(-2 kappa / A), Laplace's
law with sigma = 4 kappa phi*^2 / (3 w), phi -> -phi symmetry, the forcing
scheme's smaller spurious velocity, the diffusion of phi with mobility
Gamma (tau_phi - 1/2) and the shear-wave decay with nu = (tau - 1/2)/3; in 3D
the moments, conservation, phi -> -phi symmetry, the uniform fixed point and
the shear wave).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lb_oracle as O

C_LATTICE = O.C_LATTICE


@dataclass
class BinaryModel:
    """Parameters of a binary-fluid run: A, B, kappa (B1), Gamma (B5), tau and tau_phi (B6)."""
    lattice: str
    A: float
    B: float
    kappa: float
    Gamma: float
    tau: float
    tau_phi: float
    scheme: str = "equilibrium"      # or "forcing" (B7)
    weights: O.Weights | None = None
    stencils: O.Stencils | None = None

    def __post_init__(self):
        d = O.dim_of(self.lattice)
        if self.weights is None:
            self.weights = O.weights_d2q9() if d == 2 else O.weights_d3q19()
        if self.stencils is None:
            self.stencils = O.Stencils(dim=d)

    @property
    def dim(self):
        return O.dim_of(self.lattice)

    @property
    def e(self):
        return O.velocities(self.lattice)


# --------------------------------------------------------------------------
# Thermodynamics (B1-B3)
# --------------------------------------------------------------------------

def phi_star(A, B):
    """Bulk order parameter sqrt(-A/B) of the two phases (B1)."""
    return np.sqrt(-A / B)


def interface_width(A, kappa):
    """w of the flat profile phi* tanh(x / w): w = sqrt(-2 kappa / A) (from mu = 0, B2)."""
    return np.sqrt(-2.0 * kappa / A)


def surface_tension(A, B, kappa):
    """sigma = int kappa (dphi/dx)^2 dx over the flat profile = 4 kappa phi*^2 / (3 w)."""
    return 4.0 * kappa * phi_star(A, B) ** 2 / (3.0 * interface_width(A, kappa))


def p0(rho, phi, A, B):
    """Bulk pressure rho/3 + A/2 phi^2 + 3B/4 phi^4 (B2)."""
    return rho / 3.0 + 0.5 * A * phi ** 2 + 0.75 * B * phi ** 4


def chemical_potential(phi, lap, A, B, kappa):
    """mu = A phi + B phi^3 - kappa lap(phi) (B2)."""
    return A * phi + B * phi ** 3 - kappa * lap


def pressure_tensor(rho, phi, grad, lap, m: BinaryModel):
    """P_ab of B3 from phi's discrete gradient and Laplacian; dict (a, b) -> field."""
    d = m.dim
    g2 = sum(grad[a] ** 2 for a in range(d))
    iso = p0(rho, phi, m.A, m.B) - m.kappa * phi * lap - 0.5 * m.kappa * g2
    return {(a, b): (iso if a == b else 0.0) + m.kappa * grad[a] * grad[b] for a in range(d) for b in range(d)}


# --------------------------------------------------------------------------
# Moments and equilibria (Eq. 3, B4, B5)
# --------------------------------------------------------------------------

def moments(f: np.ndarray, g: np.ndarray, m: BinaryModel):
    """rho = sum f_i, phi = sum g_i, rho u = sum f_i e_i (Eq. 3); returns rho, phi, j, u."""
    e = m.e
    rho = f.sum(axis=0)
    phi = g.sum(axis=0)
    j = [np.einsum("i,i...->...", e[:, a].astype(np.float64), f) for a in range(m.dim)]
    u = [ja / rho for ja in j]
    return rho, phi, j, u


def _velocity_part(i, dens, u, e, w, d):
    """(w_i/c^2)(e_ia dens u_a + 3/(2c^2)[e_ia e_ib - c^2/3 d_ab] dens u_a u_b), Eq. 5 with lambda = 0."""
    c2 = C_LATTICE ** 2
    vel = sum(e[i, a] * dens * u[a] for a in range(d))
    quad = 0.0
    for a in range(d):
        for b in range(d):
            quad = quad + (e[i, a] * e[i, b] - (c2 / 3.0 if a == b else 0.0)) * dens * u[a] * u[b]
    return (w[i] / c2) * (vel + 3.0 / (2.0 * c2) * quad)


def equilibrium_f(rho, phi, u, grad, lap, m: BinaryModel, include_m_terms: bool = True):
    """f^eq of B4: Eq. 5 (i >= 1) with the binary p0 and phi's gradient terms; f_0 by Eq. 6."""
    w = m.weights
    e = m.e.astype(np.float64)
    d = m.dim
    c2 = C_LATTICE ** 2
    pres = p0(rho, phi, m.A, m.B)
    Q = len(e)
    feq = np.empty((Q,) + rho.shape)
    for i in range(1, Q):
        pr = w.wp[i] * pres - w.wt[i] * m.kappa * phi * lap
        if include_m_terms:
            for (a, b), wab in w.wm.items():
                pr = pr + wab[i] * m.kappa * grad[a] * grad[b]
        feq[i] = _velocity_part(i, rho, u, e, w.w, d) + pr / c2
    feq[0] = rho - feq[1:].sum(axis=0)
    return feq


def equilibrium_g(phi, u, mu, m: BinaryModel):
    """g^eq of B5: velocity part with phi, w^p_i Gamma mu / c^2 (i >= 1), g_0 = phi - sum."""
    w = m.weights
    e = m.e.astype(np.float64)
    d = m.dim
    c2 = C_LATTICE ** 2
    Q = len(e)
    geq = np.empty((Q,) + phi.shape)
    for i in range(1, Q):
        geq[i] = _velocity_part(i, phi, u, e, w.w, d) + w.wp[i] * m.Gamma * mu / c2
    geq[0] = phi - geq[1:].sum(axis=0)
    return geq


def body_force(phi, m: BinaryModel):
    """Body force of B7: Eq. 28 with M_ab = kappa d_a phi d_b phi."""
    return O.body_force(phi, m)


# --------------------------------------------------------------------------
# One time step and the initial state
# --------------------------------------------------------------------------

def step(f: np.ndarray, g: np.ndarray, m: BinaryModel):
    """One time step: both BGK collisions (f with tau and the force of B7, g with
    tau_phi), then streaming of both (Eq. 4).

    1. rho, phi, u (Eq. 3);  2. gradient and Laplacian of phi (B8);
    3. mu, p0 (B2);  4. f^eq (B4; without the M terms in the forcing scheme);
    5. forcing scheme: g_force (Eq. 28), F_i (Eq. 27), v (Eq. 40);  g^eq (B5,
    with v in the forcing scheme, B7);
    6. f* = f - (f - f^eq)/tau + F,  g* = g - (g - g^eq)/tau_phi; both pushed
    to r + e_i.
    """
    rho, phi, j, u = moments(f, g, m)
    grad = O.gradient(phi, m.stencils)
    lap = O.laplacian(phi, m.stencils)
    mu = chemical_potential(phi, lap, m.A, m.B, m.kappa)
    forcing = m.scheme == "forcing"
    feq = equilibrium_f(rho, phi, u, grad, lap, m, include_m_terms=not forcing)
    if forcing:
        gf = body_force(phi, m)
        F = O.force_populations(u, gf, m)
        v = [u[a] + gf[a] / (2 * rho) for a in range(m.dim)]   # Eq. 40
    else:
        F = 0.0
        v = u
    geq = equilibrium_g(phi, v, mu, m)
    fstar = f - (f - feq) / m.tau + F
    gstar = g - (g - geq) / m.tau_phi
    fo = np.empty_like(f)
    go = np.empty_like(g)
    for i, ei in enumerate(m.e):
        fo[i] = O.shift(fstar[i], -ei)
        go[i] = O.shift(gstar[i], -ei)
    return fo, go


def run(f, g, m: BinaryModel, nsteps: int):
    for _ in range(nsteps):
        f, g = step(f, g, m)
    return f, g


def drop_phi(shape, centres, radii, phi_in, phi_out, width):
    """Initial order parameter of drops of phase phi_in in phase phi_out:
    phi_out + (phi_in - phi_out) max_k 1/2 (1 + tanh((R_k - d_k) / width)),
    the tanh form of reading R12 (d_k the periodic minimum-image distance)."""
    return O.drop_density(shape, centres, radii, phi_in, phi_out, width)


def init_equilibrium(rho0, phi0, m: BinaryModel, u0=None):
    """f = f^eq, g = g^eq of (rho0, phi0, u0) (u0 = 0 by default), stencils from phi0."""
    u = u0 if u0 is not None else [np.zeros_like(rho0) for _ in range(m.dim)]
    grad = O.gradient(phi0, m.stencils)
    lap = O.laplacian(phi0, m.stencils)
    mu = chemical_potential(phi0, lap, m.A, m.B, m.kappa)
    f = equilibrium_f(rho0, phi0, u, grad, lap, m, include_m_terms=m.scheme != "forcing")
    g = equilibrium_g(phi0, u, mu, m)
    return f, g


# --------------------------------------------------------------------------
# Observables
# --------------------------------------------------------------------------

def observables(f, g, m: BinaryModel):
    """rho, phi, u (Eq. 3), v = u + g_force/(2 rho) (Eq. 40; v = u without forcing), mu (B2)."""
    rho, phi, j, u = moments(f, g, m)
    lap = O.laplacian(phi, m.stencils)
    mu = chemical_potential(phi, lap, m.A, m.B, m.kappa)
    if m.scheme == "forcing":
        gf = body_force(phi, m)
        v = [u[a] + gf[a] / (2 * rho) for a in range(m.dim)]
    else:
        v = [ua.copy() for ua in u]
    return rho, phi, u, v, mu


def diagnostics(f, g, m: BinaryModel, centre=None, far=None):
    """Mass, order-parameter total, momentum, max|u|, max|v|, and
    dP = p0 at the drop centre - p0 at a far site (B2; the gradient terms of B3
    vanish in either bulk)."""
    rho, phi, u, v, _ = observables(f, g, m)
    _, _, j, _ = moments(f, g, m)
    out = {
        "mass": float(np.sum(rho)),
        "phi_total": float(np.sum(phi)),
        "momentum": [float(np.sum(ja)) for ja in j],
        "max_u": float(np.sqrt(sum(ua ** 2 for ua in u)).max()),
        "max_v": float(np.sqrt(sum(va ** 2 for va in v)).max()),
    }
    if centre is not None and far is not None:
        out["dP"] = float(p0(rho[centre], phi[centre], m.A, m.B) - p0(rho[far], phi[far], m.A, m.B))
    return out
