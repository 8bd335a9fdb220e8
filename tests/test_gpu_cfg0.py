"""The small correctness workload over a long run: D2Q9 64^2, float64, one drop
R = 16 at (32, 32), equilibrium scheme, T = 0.55, kappa = 0.01, tau = 1.0,
5000 steps from the tanh start.  max|u| and the pressure jump dP = p0(rho at
the drop centre) - p0(rho at the far corner) (Sec. IV) every 100 steps agree
with the oracle's trajectory (R14 for u; dP, a difference of two O(1)
pressures, to 1e-12).
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from tests.helpers import A_VDW, B_VDW, library

pytestmark = pytest.mark.gpu


def test_cfg0_trajectory_matches_the_oracle():
    lb = library()
    n, R, T, kappa, tau = 64, 16.0, 0.55, 0.01, 1.0
    m = O.Model("D2Q9", A_VDW, B_VDW, T, kappa, tau, scheme="equilibrium")
    rl, rg = O.coexistence(A_VDW, B_VDW, T)
    f = O.init_equilibrium(O.drop_density((1, n, n), [(32.0, 32.0)], [R], rl, rg), m)
    with lb.Context(lb.D2Q9, (n, n), A_VDW, B_VDW, T, kappa, tau, scheme=lb.EQUILIBRIUM) as ctx:
        ctx.init_drops([(32.0, 32.0)], [R], 2.0)
        assert np.abs(ctx.get_populations() - f).max() < 1e-13
        for _ in range(50):
            ctx.step(100)
            f = O.run(f, m, 100)
            rho, u, _ = ctx.fields()
            rho = rho.reshape(n, n)
            umax = np.sqrt((u.reshape(2, -1) ** 2).sum(axis=0)).max()
            dP = O.p0(rho[32, 32], m.a, m.b, m.T) - O.p0(rho[0, 0], m.a, m.b, m.T)
            want = O.diagnostics(f, m, centre=(0, 32, 32), far=(0, 0, 0))
            assert abs(umax - want["max_u"]) <= 1e-12 * max(want["max_u"], 1e-3)
            assert abs(dP - want["dP"]) <= 1e-12        # a difference of two O(1) pressures
    assert want["max_u"] < 1e-3 and 0 < want["dP"] < 1e-2      # small flow, pressure higher inside
