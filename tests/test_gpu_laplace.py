"""Laplace's law on the CUDA path (D3Q19 and D2Q9), against the continuum surface tension.

A drop in a periodic 64^3 box at the paper's wide-interface parameters
(T = 0.56, kappa = 0.025, tau = 1, forcing scheme) relaxes for 6000 steps.
In 3D the pressure jump across a spherical interface is dP = 2 sigma / R
with sigma the planar tension of the van der Waals free energy plus
kappa/2 |grad rho|^2 (Eqs. 1-2; sigma = int sqrt(2 kappa dOmega) drho).
dP is the difference of the bulk pressures p0 (Eq. 2) inside and outside,
R the equimolar radius (3 V / 4 pi)^(1/3), V = (sum rho - rho_out N) /
(rho_in - rho_out).  The check is independent of the oracle's step: it pins
the GPU solver to a closed form.  In a closed box the drop gives mass to the
vapour until the vapour's chemical potential matches the curved interface;
below a size that depends on the box it evaporates completely (a drop of
R = 12 does in 64^3).  The interface at T = 0.56 (0.98 T_c) is several
sites wide, so small drops show the curvature correction to the law:
measured dP R / 2 sigma = 0.89 at R_e = 12.5 (R = 14 in 48^3), 0.969 at
16.4, 0.976 at 21.3.  Tolerances: the 2D oracle meets the same law within
4% at R = 20; here 5% at R = 18 (R_e 16.4), dP R constant within 3%
between R_e ~ 16 and ~ 29 (R = 30 in 96^3), the R_e 12.5 drop below both
and within 15%; the 32- and 16-bit storage formats give dP R within 1% of
float64.  D2Q9 (dP =
sigma / R, area instead of volume): a 128^2 box, R = 20 and 30, 10^4 steps,
the same bounds.
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from tests.helpers import A_VDW, B_VDW, library, sigma_continuum

pytestmark = pytest.mark.gpu

N, T, KAPPA, TAU, STEPS = 64, 0.56, 0.025, 1.0, 6000


def _laplace(storage, R, n):
    lb = library()
    with lb.Context(lb.D3Q19, (n, n, n), A_VDW, B_VDW, T, KAPPA, TAU, scheme=lb.FORCING, storage=storage) as ctx:
        ctx.init_drops([(n / 2,) * 3], [R], 2.0)
        ctx.step(STEPS)
        rho, _, _ = ctx.fields(want_v=False)
    assert np.isfinite(rho).all()
    r_in, r_out = rho[n // 2, n // 2, n // 2], rho[0, 0, 0]
    assert r_in > 1.1 * r_out     # the drop is still there
    V = (rho.sum() - r_out * rho.size) / (r_in - r_out)
    R_e = (3 * V / (4 * np.pi)) ** (1 / 3)
    dP = O.p0(r_in, A_VDW, B_VDW, T) - O.p0(r_out, A_VDW, B_VDW, T)
    return dP, R_e


_cache = {}


def laplace(storage, R, n=N):
    if (storage, R, n) not in _cache:
        _cache[(storage, R, n)] = _laplace(storage, R, n)
    return _cache[(storage, R, n)]


def test_laplace_law_3d_float64():
    sigma = sigma_continuum(T, KAPPA)
    dP, R_e = laplace(0, 18.0)
    ratio = dP * R_e / (2 * sigma)
    print(f"R_e {R_e:.3f} dP {dP:.4e} dP R / 2 sigma {ratio:.4f}")
    assert abs(ratio - 1) < 0.05, ratio


def test_laplace_pressure_scales_as_inverse_radius_3d():
    sigma = sigma_continuum(T, KAPPA)
    runs = [laplace(0, 14.0, 48), laplace(0, 18.0, 64), laplace(0, 30.0, 96)]
    r = [dP * R_e / (2 * sigma) for dP, R_e in runs]
    print("dP R / 2 sigma:", ", ".join(f"{x:.4f} (R_e {R_e:.2f})" for x, (_, R_e) in zip(r, runs)))
    assert abs(r[1] / r[2] - 1) < 0.03
    assert abs(r[2] - 1) < 0.05
    assert r[0] < min(r[1], r[2]) and abs(r[0] - 1) < 0.15


@pytest.mark.parametrize("storage", [1, 2, 3], ids=["f32", "f16dev", "bf16dev"])
def test_laplace_reduced_storage_matches_float64(storage):
    dP0, R0 = laplace(0, 18.0)
    dP, R_e = laplace(storage, 18.0)
    print(f"storage {storage}: dP R {dP * R_e:.5e} vs float64 {dP0 * R0:.5e}")
    assert abs(dP * R_e / (dP0 * R0) - 1) < 0.01


def _laplace_2d(R, n=128, steps=10000):
    lb = library()
    with lb.Context(lb.D2Q9, (n, n), A_VDW, B_VDW, T, KAPPA, TAU, scheme=lb.FORCING, storage=0) as ctx:
        ctx.init_drops([(n / 2, n / 2)], [R], 2.0)
        ctx.step(steps)
        rho, _, _ = ctx.fields(want_v=False)
    rho = rho[0]
    r_in, r_out = rho[n // 2, n // 2], rho[0, 0]
    R_e = np.sqrt((rho.sum() - r_out * rho.size) / (np.pi * (r_in - r_out)))
    dP = O.p0(r_in, A_VDW, B_VDW, T) - O.p0(r_out, A_VDW, B_VDW, T)
    return dP, R_e


def test_laplace_law_2d():
    sigma = sigma_continuum(T, KAPPA)
    dP1, R1 = _laplace_2d(20.0)
    dP2, R2 = _laplace_2d(30.0)
    print(f"2D dP R / sigma: {dP1 * R1 / sigma:.4f} (R_e {R1:.3f}), {dP2 * R2 / sigma:.4f} (R_e {R2:.3f})")
    assert abs(dP2 * R2 / sigma - 1) < 0.05
    assert abs(dP1 * R1 / (dP2 * R2) - 1) < 0.03
