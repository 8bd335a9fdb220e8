"""Shared helpers for the tests: library build, oracle models, comparisons."""
import numpy as np

from oracle import lb_oracle as O

A_VDW, B_VDW = 9.0 / 49.0, 2.0 / 21.0
LAT = {"D2Q9": 0, "D3Q19": 1}
SCHEME = {"equilibrium": 0, "forcing": 1}

_built = None


def sigma_continuum(T, kappa, a=A_VDW, b=B_VDW):
    """Planar-interface tension of psi + kappa/2 |grad rho|^2 (psi from Eq. 2):
    sigma = int_{rho_g}^{rho_l} sqrt(2 kappa (psi - mu rho + p)) drho at coexistence."""
    from scipy.integrate import quad
    rl, rg = O.coexistence(a, b, T)
    mu = O.mu0(rl, a, b, T)
    p = O.p0(rl, a, b, T)
    psi = lambda r: r * T * np.log(r / (1 - b * r)) - a * r * r - r * T
    return quad(lambda r: np.sqrt(2 * kappa * max(psi(r) - mu * r + p, 0.0)), rg, rl, limit=200)[0]


def library():
    """Build (if stale) and load liblb.so; returns the binding module."""
    global _built
    if _built is None:
        from paper_0710_5470_gb300 import build, lb
        build.build()
        lb.load_library()
        _built = lb
    return _built


def oracle_model(lat, scheme, T=0.55, kappa=0.01, tau=0.8):
    return O.Model(lat, A_VDW, B_VDW, T, kappa, tau, scheme=scheme)


def make_ctx(lb, lat, scheme, shape_xyz, storage=0, T=0.55, kappa=0.01, tau=0.8, **kw):
    return lb.Context(LAT[lat], shape_xyz, A_VDW, B_VDW, T, kappa, tau, scheme=SCHEME[scheme], storage=storage, **kw)


def drop_populations(m, shape_xyz, R, perturb=0.0, seed=0):
    """Oracle equilibrium of a centred drop, optionally perturbed (seeded noise)."""
    from paper_0710_5470_gb300 import inputs
    nx, ny, nz = (tuple(shape_xyz) + (1,))[:3]
    rl, rg = O.coexistence(m.a, m.b, m.T)
    c, r = inputs.centred_drop(shape_xyz, R)
    rho0 = O.drop_density((nz, ny, nx), c, r, rl, rg)
    f = O.init_equilibrium(rho0, m)
    if perturb:
        f = f * (1.0 + perturb * inputs.noise(seed, f.shape))
    return f


def rel_inf(a, b):
    """max |a - b| / max |b|."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
