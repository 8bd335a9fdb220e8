"""FP64 CPU oracle of the free-energy lattice Boltzmann time step.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference leg of
``bench.py``; nothing on the product path (the CUDA library in
``paper_0710_5470_gb300/`` and its Python binding) imports, calls or links it,
and it imports nothing from there.  It shares no code, table or constant with
the CUDA kernels: every lattice table below is typed in here from the paper.

Source: C. M. Pooley and K. Furtado, "Eliminating spurious velocities in the
free energy lattice Boltzmann method".  Equation numbers follow the paper
(Eq. 1 pressure tensor ... Eq. 40 fluid velocity v).  Lattice units are used
throughout: dx = dt = c = 1 (Sec. II).

Conventions
-----------
* Every field is a float64 numpy array of shape (nz, ny, nx) (nz = 1 for D2Q9),
  periodic in all directions; the site index is x + nx*(y + ny*z).
* Populations are arrays of shape (Q, nz, ny, nx).
* ``shift(a, (dx, dy, dz))`` returns a(r + (dx, dy, dz)), taken with np.roll.
* The method is written out step by step in the paper's order and notation;
  no blocking, fusion or reordering.  numpy routines (roll, sum, einsum) are
  the only library steps.

Readings where the paper is ambiguous or inconsistent (each is also listed in
the project's design notes):
* R1  Eq. 6 writes f_0 = rho - sum_i f_i; read f_i^eq (needed for Eq. 33).
* R2  Eq. 5 writes w^t rho lap(rho) without kappa; read w^t kappa rho lap(rho)
      (Eqs. 1, 14 carry kappa).
* R3  Sec. VIII lists w^xy_{5-8} = 1/4; Sec. II (after Eq. 15) gives
      w^xy_{5,6} = +1/4, w^xy_{7,8} = -1/4.  Read w^xy_i = sign(e_ix e_iy)/4,
      the only choice meeting Eq. 34.
* R4  Eq. 31 prints w_{1-6} = w^p_{1-6} = w^t_{1-6} = 1/3 for D3Q19; with
      w_{7-18} = 1/12 Eq. 34 and 2A + 8B = 1 (Eq. 29, A = 1/6) need 1/6.
      Read 1/6.
* R5  Eq. 31 prints w^xx_{1,2} = w^yy_{3,4} = w^zz_{5,6} = 1/3; Eq. 34 needs
      sum_i w^xx_i e_ix^2 = 1/2, giving 5/12.  Read 5/12.  The printed table
      stays selectable (``paper_literal=True``) so a test can show it fails.
* R6  The forcing stencil (E, F) of Eq. 28 has no stated constraint; read
      2E + 4F = 1 (2D) and 2E + 8F = 1 (3D) as for Eq. 10, so F = 1/12 gives
      the same operator as the gradient stencil (Sec. VIII).
* R7  3D forcing is not written out; read g_a = -d_b (M_ab - delta_ab M_cc/2),
      which is Eq. 28 in 2D.
* R8  The force term F_i (Eq. 27) is applied as printed (no (1 - 1/2tau)
      factor) and F_0 = -sum_{i>=1} F_i so that sum_i F_i = 0 (Eq. 37).
* R9  Eq. 5 uses the lattice velocity u of Eq. 3; the spurious velocity of the
      forcing scheme is v = u + g / (2 rho) (Eq. 40).
* R10 lambda uses the local c_s^2 = dp0/drho (Eq. 36), which may be negative
      inside the interface; its sign is kept.
* R11 The prior-art values of Sec. III (Inamuro 0, Desplat -1/72) and the
      "best choice w^p_{5-8} = -1/24" following Eq. 22 refer to w^xx_{5-8}
      (Eq. 22 must involve the M weights; Sec. VIII lists w^xx_{5-8} = -1/24).
* R12 Initial drop (synthetic workload): rho0 = rho_g + (rho_l - rho_g) *
      max_k 0.5 * (1 + tanh((R_k - d_k) / w)), with d_k the periodic minimum
      image distance of the integer site coordinates from centre k.

Parity status: every function below is pinned by ``tests/test_oracle_*.py``
(closed forms, conservation, moment identities, polynomial exactness, fold,
symmetry, Maxwell residuals, Laplace law).  The absolute size of the spurious
velocity at steady state beyond its order of magnitude (Sec. IV, Sec. VI) is
parity unpinned: the paper prints no step-level numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_LATTICE = 1.0  # c = dx/dt (Sec. II); lattice units


# --------------------------------------------------------------------------
# Velocity sets
# --------------------------------------------------------------------------

def velocities(lattice: str) -> np.ndarray:
    """Velocity vectors e_i as an (Q, 3) int array (z component 0 in 2D).

    D2Q9 (Sec. II): e_0 = 0, e_{1,2} = (+-c, 0), e_{3,4} = (0, +-c),
    e_{5,6} = (+-c, +-c), e_{7,8} = (-+c, +-c).
    D3Q19 (Sec. VII): e_{1-6} along the axes, e_{7-18} the twelve columns of
    the printed 3 x 12 matrix, in that order.
    """
    if lattice == "D2Q9":
        e = [(0, 0, 0),
             (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
             (1, 1, 0), (-1, -1, 0), (-1, 1, 0), (1, -1, 0)]
    elif lattice == "D3Q19":
        e = [(0, 0, 0),
             (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
        ex = [1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1]
        ey = [1, 1, -1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
        ez = [0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]
        e += list(zip(ex, ey, ez))
    else:
        raise ValueError(lattice)
    return np.array(e, dtype=np.int64)


def dim_of(lattice: str) -> int:
    return 2 if lattice == "D2Q9" else 3


# --------------------------------------------------------------------------
# Weights of the equilibrium distribution (Eq. 5, Sec. II-III, Eq. 31)
# --------------------------------------------------------------------------

PAIRS_2D = [(0, 0), (1, 1), (0, 1)]                          # xx, yy, xy
PAIRS_3D = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]  # xx yy zz xy yz zx


@dataclass
class Weights:
    """w_i, w^p_i, w^t_i and the M weights w^{ab}_i (one entry per pair a<=b)."""
    w: np.ndarray
    wp: np.ndarray
    wt: np.ndarray
    wm: dict = field(default_factory=dict)


def weights_d2q9(wp58: float = 1.0 / 12, wt58: float = 1.0 / 12,
                 wxx58: float = -1.0 / 24) -> Weights:
    """D2Q9 weights as functions of the three free parameters of Eq. 16.

    Velocity part: w_{1-4} = 1/3, w_{5-8} = 1/12 (after Eq. 5).
    Constraints stated after Eq. 15: 2 w^p_{1-4} + 4 w^p_{5-8} = 1, the same
    for w^t; 2 w^xx_{1-2} + 4 w^xx_{5-8} = 1/2; 2 w^yy_{1-2} + 4 w^yy_{5-8}
    = -1/2; w^xy_{1-4} = 0, w^xy_{5,6} = 1/4, w^xy_{7,8} = -1/4 (reading R3).
    Symmetries stated after Eq. 14: w^xx_{1-2} = w^yy_{3-4},
    w^xx_{3-4} = w^yy_{1-2}, w^xx_{5-8} = w^yy_{5-8}.
    The defaults are the optimum of Sec. III (listed again in Sec. VIII):
    w^p_{5-8} = w^t_{5-8} = 1/12, w^xx_{5-8} = -1/24.
    """
    w = np.array([0.0] + [1 / 3] * 4 + [1 / 12] * 4)
    wp = np.array([0.0] + [0.5 - 2 * wp58] * 4 + [wp58] * 4)
    wt = np.array([0.0] + [0.5 - 2 * wt58] * 4 + [wt58] * 4)
    wxx12 = 0.25 - 2 * wxx58
    wyy58 = wxx58
    wyy12 = -0.25 - 2 * wyy58
    wxx = np.array([0.0, wxx12, wxx12, wyy12, wyy12] + [wxx58] * 4)
    wyy = np.array([0.0, wyy12, wyy12, wxx12, wxx12] + [wyy58] * 4)
    e = velocities("D2Q9")
    wxy = np.zeros(9)
    for i in range(5, 9):
        wxy[i] = 0.25 * np.sign(e[i, 0] * e[i, 1])
    return Weights(w=w, wp=wp, wt=wt, wm={(0, 0): wxx, (1, 1): wyy, (0, 1): wxy})


def weights_d3q19(paper_literal: bool = False) -> Weights:
    """D3Q19 weights of Eq. 31 (Sec. VII), with readings R4 and R5.

    Index groups (velocity order of Sec. VII): 1,2 = +-x; 3,4 = +-y; 5,6 = +-z;
    7-10 = xy diagonals; 11-14 = yz diagonals; 15-18 = zx diagonals.
    ``paper_literal=True`` uses the printed 1/3 entries instead of the
    readings (1/6 for w_{1-6}, w^p, w^t; 5/12 for w^xx_{1,2} etc.).
    """
    face = 1 / 3 if paper_literal else 1 / 6
    self_face = 1 / 3 if paper_literal else 5 / 12
    w = np.array([0.0] + [face] * 6 + [1 / 12] * 12)
    wp = w.copy()
    wt = w.copy()
    xy = list(range(7, 11))
    yz = list(range(11, 15))
    zx = list(range(15, 19))

    def table(own_faces, other_faces, minus_edges, plus_edges):
        t = np.zeros(19)
        for i in own_faces:
            t[i] = self_face
        for i in other_faces:
            t[i] = -1 / 3
        for i in minus_edges:
            t[i] = -1 / 24
        for i in plus_edges:
            t[i] = 1 / 12
        return t

    # w^xx_{1,2} = 1/3 (R5: 5/12); w^xx_{3-6} = -1/3; w^xx_{7-10} = w^xx_{15-18}
    # = -1/24; w^xx_{11-14} = 1/12.  w^yy, w^zz by the listed permutations.
    wxx = table([1, 2], [3, 4, 5, 6], xy + zx, yz)
    wyy = table([3, 4], [1, 2, 5, 6], xy + yz, zx)
    wzz = table([5, 6], [1, 2, 3, 4], yz + zx, xy)
    # w^xy_{7,10} = w^yz_{11,14} = w^zx_{15,18} = 1/4;
    # w^xy_{8,9} = w^yz_{12,13} = w^zx_{16,17} = -1/4; all others 0.
    wxy = np.zeros(19)
    wyz = np.zeros(19)
    wzx = np.zeros(19)
    wxy[[7, 10]] = 0.25
    wxy[[8, 9]] = -0.25
    wyz[[11, 14]] = 0.25
    wyz[[12, 13]] = -0.25
    wzx[[15, 18]] = 0.25
    wzx[[16, 17]] = -0.25
    return Weights(w=w, wp=wp, wt=wt,
                   wm={(0, 0): wxx, (1, 1): wyy, (2, 2): wzz,
                       (0, 1): wxy, (1, 2): wyz, (0, 2): wzx})


# --------------------------------------------------------------------------
# Finite-difference stencils (Eqs. 10, 11, 29; optimum in Eq. 32 / Sec. VII)
# --------------------------------------------------------------------------

def shift(a: np.ndarray, off) -> np.ndarray:
    """a(r + off) on the periodic lattice; off = (dx, dy, dz)."""
    dx, dy, dz = (int(v) for v in off)
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def _matrix_offsets(mat, dz: int = 0) -> dict:
    """Offsets of a printed 3x3 stencil: top row is y = +1, left column x = -1."""
    out = {}
    for r in range(3):
        for col in range(3):
            if mat[r][col] != 0:
                out[(col - 1, 1 - r, dz)] = float(mat[r][col])
    return out


def _swap(offsets: dict, a: int, b: int) -> dict:
    """Interchange the axis labels a and b of a stencil (Sec. II, Sec. VI)."""
    out = {}
    for off, v in offsets.items():
        o = list(off)
        o[a], o[b] = o[b], o[a]
        out[tuple(o)] = v
    return out


def apply_stencil(a: np.ndarray, offsets: dict) -> np.ndarray:
    """sum over stencil entries of coefficient * a(r + offset)."""
    out = np.zeros_like(a)
    for off, coef in offsets.items():
        out += coef * shift(a, off)
    return out


@dataclass
class Stencils:
    """Coefficients of the gradient / Laplacian stencils and the force stencil.

    2D (Eqs. 10, 11): 2A + 4B = 1, C + 2D = 1; optimum B = 1/12, D = 1/6
    (Sec. III, Eq. 32).  3D (Eq. 29): 2A + 8B = 1, C + 4D = 1,
    E = -6C - 12D; A = 1/6, B = 1/12, C = 1/3, D = 1/6 (Eq. 31).  The force
    stencil (E_f, F_f) of Eq. 28 uses F_f = 1/12 (Sec. VI) and reading R6.
    """
    dim: int
    B: float = 1.0 / 12
    D: float = 1.0 / 6
    F_force: float = 1.0 / 12

    @property
    def A(self):
        return 0.5 - 2 * self.B if self.dim == 2 else (1 - 8 * self.B) / 2

    @property
    def C(self):
        return 1 - 2 * self.D if self.dim == 2 else 1 - 4 * self.D

    @property
    def E_force(self):
        return 0.5 - 2 * self.F_force if self.dim == 2 else (1 - 8 * self.F_force) / 2

    def grad_offsets(self, A=None, B=None):
        """Offsets of d_x, d_y (, d_z) as three dicts (Eq. 10 / Eq. 29)."""
        A = self.A if A is None else A
        B = self.B if B is None else B
        if self.dim == 2:
            dx = _matrix_offsets([[-B, 0, B], [-A, 0, A], [-B, 0, B]])
            return [dx, _swap(dx, 0, 1)]
        side = [[0, 0, 0], [-B, 0, B], [0, 0, 0]]
        mid = [[-B, 0, B], [-A, 0, A], [-B, 0, B]]
        dx = {}
        dx.update(_matrix_offsets(side, dz=1))
        dx.update(_matrix_offsets(mid, dz=0))
        dx.update(_matrix_offsets(side, dz=-1))
        return [dx, _swap(dx, 0, 1), _swap(dx, 0, 2)]

    def laplacian_offsets(self):
        """Offsets of the Laplacian (Eq. 11 / Eq. 29)."""
        C, D = self.C, self.D
        if self.dim == 2:
            return _matrix_offsets([[D, C, D], [C, -4 * (C + D), C], [D, C, D]])
        E = -6 * C - 12 * D
        side = [[0, D, 0], [D, C, D], [0, D, 0]]
        mid = [[D, C, D], [C, E, C], [D, C, D]]
        out = {}
        out.update(_matrix_offsets(side, dz=1))
        out.update(_matrix_offsets(mid, dz=0))
        out.update(_matrix_offsets(side, dz=-1))
        return out


def gradient(rho: np.ndarray, st: Stencils) -> list:
    """[d_x rho, d_y rho (, d_z rho)] with the stencils of Eq. 10 / Eq. 29."""
    return [apply_stencil(rho, o) for o in st.grad_offsets()]


def laplacian(rho: np.ndarray, st: Stencils) -> np.ndarray:
    """lap(rho) with the stencil of Eq. 11 / Eq. 29."""
    return apply_stencil(rho, st.laplacian_offsets())


# --------------------------------------------------------------------------
# Thermodynamics: van der Waals fluid (Eq. 2, Eq. 36) and Maxwell construction
# --------------------------------------------------------------------------

def p0(rho, a, b, T):
    """Bulk pressure p0 = rho T / (1 - b rho) - a rho^2 (Eq. 2)."""
    return rho * T / (1 - b * rho) - a * rho ** 2


def cs2(rho, a, b, T):
    """Speed of sound squared c_s^2 = dp0/drho (Eq. 36)."""
    return T / (1 - b * rho) ** 2 - 2 * a * rho


def mu0(rho, a, b, T):
    """Bulk chemical potential with p0 = rho mu0 - psi (Sec. II, Eq. 2).

    psi = rho T ln(rho / (1 - b rho)) - a rho^2 - rho T; then
    mu0 = dpsi/drho = T ln(rho / (1 - b rho)) + T b rho / (1 - b rho) - 2 a rho.
    """
    return T * np.log(rho / (1 - b * rho)) + T * b * rho / (1 - b * rho) - 2 * a * rho


def critical_point(a, b):
    """T_c = 8a / (27b), rho_c = 1 / (3b) of Eq. 2."""
    return 8 * a / (27 * b), 1 / (3 * b)


def _bisect(fun, lo, hi, iters=200):
    flo = fun(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = fun(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def coexistence(a, b, T):
    """Maxwell coexistence densities (rho_l, rho_g) of Eq. 2 below T_c.

    Liquid and gas have equal p0 and equal mu0 (the phase separation of
    Sec. II).  Plain bisection: the spinodals bound the two branches; for a
    pressure P between the spinodal pressures each branch has one density with
    p0 = P, and P is bisected until mu0(liquid) = mu0(gas).
    """
    Tc, rc = critical_point(a, b)
    if not (0 < T < Tc):
        raise ValueError("T must lie in (0, T_c)")
    f = lambda r: float(cs2(r, a, b, T))
    # spinodals: c_s^2 = 0 on either side of rho_c (c_s^2 < 0 between them)
    r_sp_g = _bisect(f, 1e-12, rc)
    r_sp_l = _bisect(f, rc, (1 - 1e-12) / b)
    p_hi = float(p0(r_sp_g, a, b, T))
    p_lo = float(p0(r_sp_l, a, b, T))
    if p_lo <= 0.0:
        # at low T the liquid spinodal pressure is negative; coexistence needs
        # P > 0, and the gas branch then runs down to rho -> 0
        p_lo = 1e-12 * p_hi

    def branches(P):
        rg = _bisect(lambda r: float(p0(r, a, b, T)) - P, 0.0, r_sp_g)
        rl = _bisect(lambda r: float(p0(r, a, b, T)) - P, r_sp_l, (1 - 1e-14) / b)
        return rl, rg

    def dmu(P):
        rl, rg = branches(P)
        return float(mu0(rl, a, b, T) - mu0(rg, a, b, T))

    P = _bisect(dmu, p_lo, p_hi)
    return branches(P)


# --------------------------------------------------------------------------
# Moments, equilibrium and forcing (Eqs. 3, 5, 6, 27, 28, 36)
# --------------------------------------------------------------------------

@dataclass
class Model:
    """Parameters of one run (Sec. IV): van der Waals a, b, T; kappa; tau."""
    lattice: str
    a: float
    b: float
    T: float
    kappa: float
    tau: float
    scheme: str = "equilibrium"      # or "forcing" (Sec. VI)
    weights: Weights | None = None
    stencils: Stencils | None = None

    def __post_init__(self):
        d = dim_of(self.lattice)
        if self.weights is None:
            self.weights = weights_d2q9() if d == 2 else weights_d3q19()
        if self.stencils is None:
            self.stencils = Stencils(dim=d)

    @property
    def dim(self):
        return dim_of(self.lattice)

    @property
    def e(self):
        return velocities(self.lattice)


def moments(f: np.ndarray, m: Model):
    """rho = sum_i f_i, rho u_a = sum_i f_i e_ia (Eq. 3); returns rho, j, u."""
    e = m.e
    rho = f.sum(axis=0)
    j = [np.einsum("i,i...->...", e[:, a].astype(np.float64), f) for a in range(m.dim)]
    u = [ja / rho for ja in j]
    return rho, j, u


def galilean_lambda(rho, m: Model):
    """nu = (tau - 1/2)/3 and lambda = nu (1 - 3 c_s^2 / c^2) (Eq. 36)."""
    nu = (m.tau - 0.5) / 3.0
    return nu * (1 - 3 * cs2(rho, m.a, m.b, m.T) / C_LATTICE ** 2)


def equilibrium(rho, u, grad, lap, m: Model, include_m_terms: bool = True):
    """Equilibrium distribution, Eq. 5 for i >= 1 and Eq. 6 for i = 0.

    For i >= 1:
      f_i^eq = (w_i/c^2) ( e_ia rho u_a + 3/(2c^2) [e_ia e_ib - c^2/3 d_ab] *
               (rho u_a u_b + lambda [u_a d_b rho + u_b d_a rho + d_ab u_g d_g rho]) )
             + (1/c^2) ( w^p_i p0 - w^t_i kappa rho lap(rho)          (R2)
                         + sum_{a<=b} w^ab_i kappa d_a rho d_b rho )
    The M_ab = kappa d_a rho d_b rho terms are dropped in the forcing scheme
    (Sec. VI).  f_0^eq = rho - sum_{i>=1} f_i^eq (Eq. 6, reading R1).
    """
    w = m.weights
    e = m.e.astype(np.float64)
    d = m.dim
    c2 = C_LATTICE ** 2
    lam = galilean_lambda(rho, m)
    pres = p0(rho, m.a, m.b, m.T)
    udotg = sum(u[g] * grad[g] for g in range(d))
    # the symmetric tensor in round brackets of Eq. 5
    S = {}
    for a_ in range(d):
        for b_ in range(d):
            S[(a_, b_)] = rho * u[a_] * u[b_] + lam * (
                u[a_] * grad[b_] + u[b_] * grad[a_] + (1.0 if a_ == b_ else 0.0) * udotg)
    Q = len(e)
    feq = np.empty((Q,) + rho.shape)
    for i in range(1, Q):
        vel = sum(e[i, a_] * rho * u[a_] for a_ in range(d))
        quad = 0.0
        for a_ in range(d):
            for b_ in range(d):
                quad = quad + (e[i, a_] * e[i, b_] - (c2 / 3.0 if a_ == b_ else 0.0)) * S[(a_, b_)]
        val = (w.w[i] / c2) * (vel + 3.0 / (2.0 * c2) * quad)
        pr = w.wp[i] * pres - w.wt[i] * m.kappa * rho * lap
        if include_m_terms:
            for (a_, b_), wab in w.wm.items():
                pr = pr + wab[i] * m.kappa * grad[a_] * grad[b_]
        feq[i] = val + pr / c2
    feq[0] = rho - feq[1:].sum(axis=0)
    return feq


def body_force(rho, m: Model):
    """Body force g of the forcing scheme (Sec. VI, Eq. 28).

    M_ab = kappa d_a rho d_b rho with the gradient stencil; then, in 2D,
      g_x = -1/2 d_x (M_xx - M_yy) - d_y M_xy,
      g_y = -1/2 d_y (M_yy - M_xx) - d_x M_xy
    ("interchanging the labels x and y"), both with the force stencil (E, F).
    In 3D (reading R7): g_a = -sum_b d_b (M_ab - delta_ab (M_xx+M_yy+M_zz)/2).
    """
    st = m.stencils
    grad = gradient(rho, st)
    d = m.dim
    M = {(a_, b_): m.kappa * grad[a_] * grad[b_] for a_ in range(d) for b_ in range(d)}
    fd = [apply_stencil_factory(st, a_) for a_ in range(d)]
    if d == 2:
        gx = -0.5 * fd[0](M[(0, 0)] - M[(1, 1)]) - fd[1](M[(0, 1)])
        gy = -0.5 * fd[1](M[(1, 1)] - M[(0, 0)]) - fd[0](M[(0, 1)])
        return [gx, gy]
    trM = M[(0, 0)] + M[(1, 1)] + M[(2, 2)]
    g = []
    for a_ in range(3):
        acc = np.zeros_like(rho)
        for b_ in range(3):
            acc = acc + fd[b_](M[(a_, b_)] - (0.5 * trM if a_ == b_ else 0.0))
        g.append(-acc)
    return g


def apply_stencil_factory(st: Stencils, axis: int):
    """Derivative along ``axis`` with the force stencil (E_f, F_f) of Eq. 28."""
    offs = st.grad_offsets(A=st.E_force, B=st.F_force)[axis]
    return lambda a: apply_stencil(a, offs)


def force_populations(u, g, m: Model):
    """F_i of Eq. 27 for i >= 1 and F_0 = -sum_{i>=1} F_i (reading R8).

    F_i = (w_i/c^2) ( e_ia g_a + 3/(2c^2) [e_ia e_ib - c^2/3 d_ab] (u_a g_b + u_b g_a) ).
    """
    e = m.e.astype(np.float64)
    w = m.weights.w
    d = m.dim
    c2 = C_LATTICE ** 2
    Q = len(e)
    F = np.empty((Q,) + u[0].shape)
    for i in range(1, Q):
        lin = sum(e[i, a_] * g[a_] for a_ in range(d))
        quad = 0.0
        for a_ in range(d):
            for b_ in range(d):
                quad = quad + (e[i, a_] * e[i, b_] - (c2 / 3.0 if a_ == b_ else 0.0)) * (
                    u[a_] * g[b_] + u[b_] * g[a_])
        F[i] = (w[i] / c2) * (lin + 3.0 / (2.0 * c2) * quad)
    F[0] = -F[1:].sum(axis=0)
    return F


# --------------------------------------------------------------------------
# One time step (Eq. 4) and the initial state
# --------------------------------------------------------------------------

def step(f: np.ndarray, m: Model) -> np.ndarray:
    """One time step of Eq. 4: BGK collision with optional force, then streaming.

    1. rho, u from Eq. 3;  2. stencils Eq. 10/11 (Eq. 29 in 3D);
    3. p0 (Eq. 2), lambda (Eq. 36);  4. f^eq (Eqs. 5, 6), without the M terms
    in the forcing scheme;  5. forcing scheme: g (Eq. 28), F_i (Eq. 27);
    6. f*_i = f_i - (f_i - f_i^eq)/tau + F_i, then f_i(r + e_i, t+1) = f*_i(r).
    """
    rho, j, u = moments(f, m)
    grad = gradient(rho, m.stencils)
    lap = laplacian(rho, m.stencils)
    forcing = m.scheme == "forcing"
    feq = equilibrium(rho, u, grad, lap, m, include_m_terms=not forcing)
    if forcing:
        g = body_force(rho, m)
        F = force_populations(u, g, m)
    else:
        F = 0.0
    fstar = f - (f - feq) / m.tau + F
    out = np.empty_like(f)
    for i, ei in enumerate(m.e):
        out[i] = shift(fstar[i], -ei)   # value at r comes from r - e_i
    return out


def run(f: np.ndarray, m: Model, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        f = step(f, m)
    return f


def drop_density(shape, centres, radii, rho_l, rho_g, width=2.0):
    """Initial density of one or more drops (reading R12).

    rho0 = rho_g + (rho_l - rho_g) * max_k 1/2 (1 + tanh((R_k - d_k)/width)),
    d_k the periodic minimum-image distance of the integer site coordinates
    from centre k.  ``shape`` is (nz, ny, nx); centres are (x, y[, z]).
    """
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)]
    sizes = [nx, ny, nz]
    prof = np.zeros(shape)
    for c, R in zip(centres, radii):
        d2 = np.zeros(shape)
        for a_ in range(len(c)):
            dd = np.abs(coords[a_] - c[a_])
            dd = np.minimum(dd, sizes[a_] - dd)
            d2 += dd ** 2
        prof = np.maximum(prof, 0.5 * (1 + np.tanh((R - np.sqrt(d2)) / width)))
    return rho_g + (rho_l - rho_g) * prof


def init_equilibrium(rho0: np.ndarray, m: Model) -> np.ndarray:
    """f = f^eq(rho0, u = 0) of the chosen scheme, stencils from rho0 (Eq. 5)."""
    zero = [np.zeros_like(rho0) for _ in range(m.dim)]
    grad = gradient(rho0, m.stencils)
    lap = laplacian(rho0, m.stencils)
    return equilibrium(rho0, zero, grad, lap, m, include_m_terms=m.scheme != "forcing")


# --------------------------------------------------------------------------
# Observables (Sec. IV, Eq. 40)
# --------------------------------------------------------------------------

def observables(f: np.ndarray, m: Model):
    """rho, u (Eq. 3) and v = u + g/(2 rho) (Eq. 40; v = u without forcing)."""
    rho, j, u = moments(f, m)
    if m.scheme == "forcing":
        g = body_force(rho, m)
        v = [u[a_] + g[a_] / (2 * rho) for a_ in range(m.dim)]
    else:
        v = [ua.copy() for ua in u]
    return rho, u, v


def diagnostics(f: np.ndarray, m: Model, centre=None, far=None):
    """Total mass and momentum, max|u|, max|v| (Sec. IV: maximum velocity
    magnitude), and dP = p0(rho at centre) - p0(rho at far site)."""
    rho, u, v = observables(f, m)
    _, j, _ = moments(f, m)
    out = {
        "mass": float(np.sum(rho)),
        "momentum": [float(np.sum(ja)) for ja in j],
        "max_u": float(np.sqrt(sum(ua ** 2 for ua in u)).max()),
        "max_v": float(np.sqrt(sum(va ** 2 for va in v)).max()),
    }
    if centre is not None and far is not None:
        cz, cy, cx = centre
        fz, fy, fx = far
        out["dP"] = float(p0(rho[cz, cy, cx], m.a, m.b, m.T) - p0(rho[fz, fy, fx], m.a, m.b, m.T))
    return out
