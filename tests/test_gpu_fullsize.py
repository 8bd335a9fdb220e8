"""Parity at the bench workload's full size, in the launch configuration bench.py times.

D3Q19 128^3, one centred drop R = 30 (tanh width 2), forcing scheme (and the
equilibrium scheme of bench.py's equilibrium block), T = 0.55, kappa = 0.01,
tau = 1.0: the library chooses the kernel, tile, z chunk (one wave of CTAs)
and layout from the size exactly as for the bench.
The oracle takes one whole step of the 128^3 lattice (a few seconds on the
host) from the GPU's own state after 20 steps, decoded to float64, and every
population of the GPU's next step is compared with it.
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from tests.helpers import A_VDW, B_VDW, library, rel_inf

pytestmark = pytest.mark.gpu

N, R = 128, 30.0
T, KAPPA, TAU = 0.55, 0.01, 1.0
# storage -> bound on max|f_gpu - f_oracle| / max|f_oracle| after one step
TOL = {0: 1e-12, 1: 2e-6, 2: 1e-4, 3: 1e-3}


@pytest.mark.parametrize("scheme", ["forcing", "equilibrium"])
@pytest.mark.parametrize("storage", [0, 1, 2, 3], ids=["f64", "f32", "f16dev", "bf16dev"])
def test_one_step_parity_at_128_cubed(storage, scheme):
    lb = library()
    m = O.Model("D3Q19", A_VDW, B_VDW, T, KAPPA, TAU, scheme=scheme)
    sch = lb.FORCING if scheme == "forcing" else lb.EQUILIBRIUM
    with lb.Context(lb.D3Q19, (N, N, N), A_VDW, B_VDW, T, KAPPA, TAU, scheme=sch, storage=storage) as ctx:
        ctx.init_drops([(N / 2,) * 3], [R], 2.0)
        ctx.step(20)
        start = ctx.get_populations()
        ctx.step(1)
        got = ctx.get_populations()
    want = O.step(start, m)
    err = rel_inf(got, want)
    assert np.isfinite(got).all()
    assert err < TOL[storage], err
