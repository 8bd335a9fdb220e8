"""The oracles' pins catch plausible mistakes planted into the oracles (on the CPU).

Each case plants one slip - a dropped term, a wrong sign, a transposed index, a
wrong velocity - into a copy or a parameter of an oracle, reruns the check a pin
makes, and asserts that the check fails.  A pin that passed with the mistake in
place would not be pinning the oracle to anything.
"""
import numpy as np
import pytest

from oracle import binary_oracle as BO
from oracle import lb_oracle as O
from tests.test_binary_oracle import _model, thermodynamic_residual, A_BIN, K_BIN
from tests.test_oracle_pins import A_VDW, B_VDW, _pressure_tensor, _random_state, eq28_error, galilean_errors


def _second_moment_error(weights, cs2_sign=1.0):
    """Max error of sum f^eq e_a e_b against P + rho u u + lambda(...) (Eq. 34), as in
    test_equilibrium_moments, for D2Q9 with the given weights."""
    rng = np.random.default_rng(3)
    m = O.Model("D2Q9", A_VDW, B_VDW, 0.55, 0.01, 0.8, weights=weights)
    rho, u, grad, lap = _random_state("D2Q9", rng)
    feq = O.equilibrium(rho, u, grad, lap, m)
    e = m.e.astype(float)
    P = _pressure_tensor(rho, grad, lap, m)
    lam = (m.tau - 0.5) / 3 * (1 - 3 * cs2_sign * O.cs2(rho, m.a, m.b, m.T))
    udg = u[0] * grad[0] + u[1] * grad[1]
    err = 0.0
    for a in range(2):
        for b in range(2):
            got = np.einsum("i,i,i...->...", e[:, a], e[:, b], feq)
            want = P[(a, b)] + rho * u[a] * u[b] + lam * (u[a] * grad[b] + u[b] * grad[a] + (a == b) * udg)
            err = max(err, float(np.abs(got - want).max()))
    return err


def test_correct_weights_pass_the_moment_check():
    assert _second_moment_error(O.weights_d2q9()) < 1e-12


def test_dropped_laplacian_term_is_caught():
    """w^t_i kappa rho lap(rho) left out of Eq. 5 (the kappa of reading R2 and more)."""
    w = O.weights_d2q9()
    w.wt = np.zeros_like(w.wt)
    assert _second_moment_error(w) > 1e-3


def test_wrong_sign_of_the_xy_weights_is_caught():
    """w^xy_{5-8} = +1/4 for all four diagonals (the misreading reading R3 avoids)."""
    w = O.weights_d2q9()
    w.wm[(0, 1)] = np.abs(w.wm[(0, 1)])
    assert _second_moment_error(w) > 1e-3


def test_transposed_m_weights_are_caught():
    """w^xx and w^yy exchanged (a transposed tensor index)."""
    w = O.weights_d2q9()
    w.wm[(0, 0)], w.wm[(1, 1)] = w.wm[(1, 1)].copy(), w.wm[(0, 0)].copy()
    assert _second_moment_error(w) > 1e-3


def test_wrong_sign_of_the_sound_speed_in_lambda_is_caught():
    """The oracle's lambda compared against nu (1 + 3 c_s^2): Eq. 36 with a sign slip."""
    assert _second_moment_error(O.weights_d2q9(), cs2_sign=-1.0) > 1e-4


def test_reversed_streaming_is_caught():
    """Populations pushed to r - e_i instead of r + e_i: the drop no longer moves with the flow."""
    def backwards(f, m):
        rho, j, u = O.moments(f, m)
        grad, lap = O.gradient(rho, m.stencils), O.laplacian(rho, m.stencils)
        forcing = m.scheme == "forcing"
        feq = O.equilibrium(rho, u, grad, lap, m, include_m_terms=not forcing)
        F = O.force_populations(u, O.body_force(rho, m), m) if forcing else 0.0
        fstar = f - (f - feq) / m.tau + F
        return np.stack([O.shift(fstar[i], tuple(ei)) for i, ei in enumerate(m.e)])
    fwd, _ = galilean_errors(step=backwards)
    assert fwd > 0.15, fwd


def test_wrong_binary_bulk_pressure_is_caught():
    """p0 = rho/3 + A phi^2 + 3B/4 phi^4 (the 1/2 of B2 dropped)."""
    assert thermodynamic_residual(p0_fn=lambda r, f, A, B: r / 3 + A * f ** 2 + 0.75 * B * f ** 4) > 1e-3


def test_wrong_sign_in_the_chemical_potential_is_caught():
    """mu = A phi + B phi^3 + kappa lap(phi)."""
    assert thermodynamic_residual(mu_fn=lambda f, l, A, B, k: A * f + B * f ** 3 + k * l) > 1e-4


def test_order_parameter_advected_with_u_in_the_forcing_scheme_is_caught():
    """g^eq with the lattice velocity u instead of the fluid velocity v of Eq. 40
    (reading B7): a flat interface then drifts off its profile and mu stays large."""
    m = _model("forcing")

    def step_u(f, g, m):
        rho, phi, j, u = BO.moments(f, g, m)
        grad, lap = O.gradient(phi, m.stencils), O.laplacian(phi, m.stencils)
        mu = BO.chemical_potential(phi, lap, m.A, m.B, m.kappa)
        feq = BO.equilibrium_f(rho, phi, u, grad, lap, m, include_m_terms=False)
        F = O.force_populations(u, BO.body_force(phi, m), m)
        geq = BO.equilibrium_g(phi, u, mu, m)
        fs, gs = f - (f - feq) / m.tau + F, g - (g - geq) / m.tau_phi
        return (np.stack([O.shift(fs[i], tuple(-ei)) for i, ei in enumerate(m.e)]),
                np.stack([O.shift(gs[i], tuple(-ei)) for i, ei in enumerate(m.e)]))

    nx, ny = 64, 4
    x = np.arange(nx, dtype=np.float64)[None, None, :] * np.ones((1, ny, 1))
    w = BO.interface_width(A_BIN, K_BIN)
    phi0 = np.tanh((x - 16) / w) - np.tanh((x - 48) / w) - 1.0
    f, g = BO.init_equilibrium(np.ones_like(phi0), phi0, m)
    for _ in range(800):
        f, g = step_u(f, g, m)
    mu = BO.observables(f, g, m)[4]
    assert np.abs(mu).max() > 1e-3      # the pin asks |mu| < 1e-4


def test_wrong_sign_or_transposed_body_force_is_caught():
    """g = +div M' instead of -div M' (Eq. 28), or its components exchanged."""
    assert eq28_error(lambda rho, m: [-c for c in O.body_force(rho, m)]) > 1e-6
    assert eq28_error(lambda rho, m: O.body_force(rho, m)[::-1]) > 1e-6
