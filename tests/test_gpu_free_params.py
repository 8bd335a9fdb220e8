"""The D2Q9 step with run-time free parameters (lb_set_free_params) against the oracle.

The oracle takes the same free parameters (weights_d2q9(w^p_{5-8}, w^t_{5-8},
w^xx_{5-8}), Stencils(2, B, D, F)); the library derives the other weights
and stencil coefficients on its own from the constraints of Secs. II-III.
Parity is element by element to 1e-12 (float64), for parameter sets away
from the optimum (the Fig. 2 scans and the prior-art choices of Sec. III).
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from paper_0710_5470_gb300 import inputs
from tests.helpers import A_VDW, B_VDW, library, make_ctx, rel_inf

pytestmark = pytest.mark.gpu

# (w^p_58, w^t_58, w^xx_58, B, D, F)
SETS = {
    "inamuro_wxx": (1 / 12, 1 / 12, 0.0, 1 / 12, 1 / 6, 1 / 12),
    "desplat_wxx": (1 / 12, 1 / 12, -1 / 72, 1 / 12, 1 / 6, 1 / 12),
    "gradient_B0": (1 / 12, 1 / 12, -1 / 24, 0.0, 1 / 6, 1 / 12),      # the B = 0 point of Fig. 2(b)
    "all_off": (0.05, 0.11, -0.02, 0.1, 0.2, 0.06),
}


def model(scheme, p, T=0.56, kappa=0.025, tau=0.9):
    wp, wt, wxx, B, D, F = p
    return O.Model("D2Q9", A_VDW, B_VDW, T, kappa, tau, scheme=scheme, weights=O.weights_d2q9(wp, wt, wxx),
                   stencils=O.Stencils(2, B=B, D=D, F_force=F))


def kw(p):
    return dict(zip(("wp58", "wt58", "wxx58", "B", "D", "F"), p))


def drop_state(m, shape, R, perturb, seed):
    nx, ny = shape
    rl, rg = O.coexistence(m.a, m.b, m.T)
    c, r = inputs.centred_drop(shape, R)
    f = O.init_equilibrium(O.drop_density((1, ny, nx), c, r, rl, rg), m)
    return f * (1.0 + perturb * inputs.noise(seed, f.shape))


@pytest.mark.parametrize("name", list(SETS))
@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_free_parameter_step_parity(scheme, name):
    lb = library()
    p = SETS[name]
    m = model(scheme, p)
    shape = (45, 37)
    f0 = drop_state(m, shape, 11.0, 1e-3, 4)
    with make_ctx(lb, "D2Q9", scheme, shape, T=m.T, kappa=m.kappa, tau=m.tau) as ctx:
        ctx.set_free_params(**kw(p))
        ctx.set_populations(f0)
        ctx.step(40)
        got = ctx.get_populations()
        rho, u, v = ctx.fields()
    want = O.run(f0, m, 40)
    assert rel_inf(got, want) < 1e-12
    rho_o, u_o, v_o = O.observables(want, m)
    v_o = np.stack(v_o)
    assert rel_inf(rho.reshape(rho_o.shape), rho_o) < 1e-12
    vmax = max(np.abs(v_o).max(), 1e-3)
    assert np.abs(v.reshape(v_o.shape) - v_o).max() < 1e-12 * vmax


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_free_parameter_init_parity(scheme):
    lb = library()
    p = SETS["all_off"]
    m = model(scheme, p)
    shape = (40, 34)
    rl, rg = O.coexistence(m.a, m.b, m.T)
    with make_ctx(lb, "D2Q9", scheme, shape, T=m.T, kappa=m.kappa, tau=m.tau) as ctx:
        ctx.set_free_params(**kw(p))
        ctx.init_drops([(20.0, 17.0)], [9.0])
        got = ctx.get_populations()
    want = O.init_equilibrium(O.drop_density((1, 34, 40), [(20.0, 17.0)], [9.0], rl, rg), m)
    assert rel_inf(got, want) < 1e-12


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_optimum_free_parameters_reproduce_the_fused_kernel(scheme):
    lb = library()
    shape = (64, 48)
    runs = []
    for free in (False, True):
        with make_ctx(lb, "D2Q9", scheme, shape, T=0.56, kappa=0.025, tau=1.0) as ctx:
            if free:
                ctx.set_free_params()
            ctx.init_drops([(32.0, 24.0)], [14.0])
            ctx.step(200)
            runs.append(ctx.get_populations())
    assert rel_inf(runs[1], runs[0]) < 1e-12


def test_free_parameters_need_d2q9_float64():
    lb = library()
    with make_ctx(lb, "D3Q19", "forcing", (8, 8, 8)) as ctx:
        with pytest.raises(lb.LBError):
            ctx.set_free_params()
    with make_ctx(lb, "D2Q9", "forcing", (8, 8), storage=1) as ctx:
        with pytest.raises(lb.LBError):
            ctx.set_free_params()
    with make_ctx(lb, "D2Q9", "forcing", (8, 8)) as ctx:
        with pytest.raises(lb.LBError):
            ctx.set_free_params(B=float("nan"))
        ctx.set_free_params(B=0.0)
        ctx.clear_free_params()
