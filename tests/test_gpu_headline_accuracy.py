"""Accuracy of the reduced storage formats at the headline workload, against
the stated mixed-precision bounds: D3Q19 128^3, one centred drop R = 30, forcing scheme,
T = 0.55, kappa = 0.01, tau = 1, 10^4 steps from the tanh start, each format
compared with the float64 path (which matches the oracle to 1e-12 per step
on smaller lattices; the oracle itself would need hours here).

Bounds: the spurious velocity max|v| (Eq. 40) within 5%, and
rho within 1e-5 relative.  The density bound is tested on two quantities:
the bulk densities (the extremes of rho, the liquid and vapour values), which
every format meets, and rho site by site, which no float32 arithmetic meets
(float32 storage included): the drop's radius is set by the Laplace pressure
jump (~1.3e-3 here), about 500 times smaller than p0 (~0.64), so float32
rounding of the equation of state (of T, a, b themselves and of p0) moves
the interface by ~1e-3 of a site, i.e. ~1e-3 in rho at the interface.  Those
are kept at 1e-5 and marked as expected failures; the test also
checks that the error is not a translation of the drop (the measured drift
is below 1e-2 sites) and that it does not come from the 16-bit storage (the
16-bit formats stay within 2x of float32 storage).
"""
import numpy as np
import pytest

from tests.helpers import library

pytestmark = pytest.mark.gpu

STEPS = 10000
FORMATS = ("f32", "f16dev", "bf16dev")
POINTWISE_REASON = ("float32 arithmetic moves the interface: pointwise rho error ~1e-3 (float32 storage "
                    "included), above the 1e-5 bound")


@pytest.fixture(scope="module")
def runs():
    lb = library()
    from paper_0710_5470_gb300 import accuracy as A
    rl, rg = lb.coexistence(A.A_VDW, A.B_VDW, 0.55)
    rho0, v0, _ = A.run("f64", 128, STEPS)
    out = {}
    for s in FORMATS:
        rho, v, _ = A.run(s, 128, STEPS)
        out[s] = A.compare(rho0, v0, rho, v, rl, rg)
    return out


@pytest.mark.parametrize("storage", FORMATS)
def test_spurious_velocity_within_5_percent(runs, storage):
    assert runs[storage]["max_v_rel_err"] < 0.05


@pytest.mark.parametrize("storage", FORMATS)
def test_bulk_densities_within_1e5(runs, storage):
    assert runs[storage]["rho_extremes_rel_err"] < 1e-5


@pytest.mark.parametrize("storage", [pytest.param(s, marks=pytest.mark.xfail(strict=True, reason=POINTWISE_REASON))
                                     for s in FORMATS])
def test_pointwise_density_within_1e5(runs, storage):
    assert runs[storage]["rho_pointwise_rel_err"] < 1e-5


@pytest.mark.parametrize("storage", FORMATS)
def test_density_error_is_neither_drift_nor_storage(runs, storage):
    r = runs[storage]
    assert max(abs(d) for d in r["drift_sites"]) < 1e-2
    assert r["rho_pointwise_rel_err"] < 2.0 * runs["f32"]["rho_pointwise_rel_err"] + 1e-6
    assert r["rho_pointwise_rel_err"] < 1e-2
