"""Pins of the binary-fluid oracle (oracle/binary_oracle.py, readings B1-B8).

Each pin checks the oracle against something other than itself:
* the textbook D2Q9 equilibrium w_i rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2)
  (standard weights 4/9, 1/9, 1/36) when the free energy reduces to an ideal
  gas (f) or to a passive scalar with Gamma mu = phi / 3 (g);
* the moments of f^eq and g^eq against the closed forms of B3 and B5;
* exact conservation of mass, order parameter and momentum;
* the phi -> -phi symmetry of the free energy (B1: psi even in phi);
* the flat interface phi* tanh(x / w), w = sqrt(-2 kappa / A): mu = 0 in the
  continuum, so the lattice profile stays close to it with small velocities;
* Laplace's law dP = sigma / R in 2D with sigma = 4 kappa phi*^2 / (3 w);
* the forcing scheme's smaller spurious velocity (Sec. VI, carried over by B7);
* the diffusion of phi with mobility Gamma (tau_phi - 1/2) and the decay of a
  shear wave with nu = (tau - 1/2)/3 (textbook BGK closed forms).
"""
import numpy as np
import pytest

from oracle import binary_oracle as BO
from oracle import lb_oracle as O
from paper_0710_5470_gb300 import inputs

A_BIN, B_BIN, K_BIN = -0.04, 0.04, 0.08     # phi* = 1, w = 2
W_STD = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}      # textbook D2Q9 weights by |e|^2


def _model(scheme="equilibrium", A=A_BIN, B=B_BIN, kappa=K_BIN, Gamma=1.0, tau=1.0, tau_phi=1.0):
    return BO.BinaryModel("D2Q9", A, B, kappa, Gamma, tau, tau_phi, scheme=scheme)


def _smooth_fields(n=12, seed=3):
    """Smooth periodic rho ~ 1, phi in (-1, 1), u ~ 0.05 on an n x n lattice."""
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = 2 * np.pi / n
    r = inputs.noise(seed, (6,))
    rho = (1.0 + 0.05 * np.sin(k * x + r[0]) * np.cos(k * y + r[1]))[None]
    phi = (0.8 * np.sin(k * x + r[2]) + 0.1 * np.cos(2 * k * y + r[3]))[None]
    u = [(0.05 * np.cos(k * y + r[4]))[None], (0.04 * np.sin(k * x + r[5]))[None]]
    return rho, phi, u


def _textbook(dens, u):
    e = O.velocities("D2Q9").astype(np.float64)
    usq = u[0] ** 2 + u[1] ** 2
    out = []
    for i in range(9):
        eu = e[i, 0] * u[0] + e[i, 1] * u[1]
        out.append(W_STD[int(e[i] @ e[i])] * dens * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * usq))
    return np.array(out)


def test_f_equilibrium_reduces_to_textbook_ideal_gas():
    """A = B = kappa = 0: p0 = rho/3 and no gradient terms; f^eq is the textbook D2Q9 equilibrium."""
    m = _model(A=0.0, B=0.0, kappa=0.0)
    rho, phi, u = _smooth_fields()
    grad = O.gradient(phi, m.stencils)
    lap = O.laplacian(phi, m.stencils)
    feq = BO.equilibrium_f(rho, phi, u, grad, lap, m)
    assert np.abs(feq - _textbook(rho, u)).max() < 1e-15


def test_g_equilibrium_reduces_to_textbook_passive_scalar():
    """B = kappa = 0 and A = 1/(3 Gamma): Gamma mu = phi/3, and g^eq is the textbook
    equilibrium with phi as the density."""
    Gamma = 0.7
    m = _model(A=1.0 / (3 * Gamma), B=0.0, kappa=0.0, Gamma=Gamma)
    rho, phi, u = _smooth_fields()
    lap = O.laplacian(phi, m.stencils)
    mu = BO.chemical_potential(phi, lap, m.A, m.B, m.kappa)
    geq = BO.equilibrium_g(phi, u, mu, m)
    assert np.abs(geq - _textbook(phi, u)).max() < 1e-15


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_f_equilibrium_moments_match_pressure_tensor(scheme):
    """sum f = rho, sum f e = rho u, sum f e_a e_b = P_ab + rho u_a u_b (B3); the forcing
    scheme's f^eq lacks the M part kappa (d_a phi d_b phi - |grad phi|^2 d_ab / 2) (B7)."""
    m = _model(scheme)
    rho, phi, u = _smooth_fields()
    grad = O.gradient(phi, m.stencils)
    lap = O.laplacian(phi, m.stencils)
    feq = BO.equilibrium_f(rho, phi, u, grad, lap, m, include_m_terms=scheme == "equilibrium")
    e = m.e.astype(np.float64)
    g2 = grad[0] ** 2 + grad[1] ** 2
    for a in range(2):
        assert np.abs(np.einsum("i,i...->...", e[:, a], feq) - rho * u[a]).max() < 1e-15
        for b in range(2):
            mom2 = np.einsum("i,i,i...->...", e[:, a], e[:, b], feq)
            P = (BO.p0(rho, phi, m.A, m.B) - m.kappa * phi * lap - 0.5 * m.kappa * g2) * (a == b) \
                + m.kappa * grad[a] * grad[b]
            if scheme == "forcing":
                P = P - m.kappa * (grad[a] * grad[b] - 0.5 * g2 * (a == b))
            assert np.abs(mom2 - (P + rho * u[a] * u[b])).max() < 1e-14, (a, b)
    assert np.abs(feq.sum(axis=0) - rho).max() < 1e-15


def test_g_equilibrium_moments():
    """sum g = phi, sum g e = phi u, sum g e_a e_b = Gamma mu d_ab + phi u_a u_b (B5),
    mu = A phi + B phi^3 - kappa lap(phi) (B2)."""
    m = _model(Gamma=0.6)
    rho, phi, u = _smooth_fields()
    lap = O.laplacian(phi, m.stencils)
    mu = m.A * phi + m.B * phi ** 3 - m.kappa * lap
    geq = BO.equilibrium_g(phi, u, BO.chemical_potential(phi, lap, m.A, m.B, m.kappa), m)
    e = m.e.astype(np.float64)
    assert np.abs(geq.sum(axis=0) - phi).max() < 1e-15
    for a in range(2):
        assert np.abs(np.einsum("i,i...->...", e[:, a], geq) - phi * u[a]).max() < 1e-15
        for b in range(2):
            mom2 = np.einsum("i,i,i...->...", e[:, a], e[:, b], geq)
            want = m.Gamma * mu * (a == b) + phi * u[a] * u[b]
            assert np.abs(mom2 - want).max() < 1e-15


def test_closed_forms_of_the_flat_interface():
    """phi* tanh(x / w) solves A phi + B phi^3 - kappa phi'' = 0, and sigma = int kappa phi'^2 dx."""
    from scipy.integrate import quad
    ps, w = BO.phi_star(A_BIN, B_BIN), BO.interface_width(A_BIN, K_BIN)
    x = np.linspace(-10, 10, 2001)
    phi = ps * np.tanh(x / w)
    d2 = -2 * ps / w ** 2 * np.tanh(x / w) / np.cosh(x / w) ** 2
    assert np.abs(A_BIN * phi + B_BIN * phi ** 3 - K_BIN * d2).max() < 1e-15
    sig = quad(lambda s: K_BIN * (ps / w / np.cosh(s / w) ** 2) ** 2, -60, 60)[0]
    assert abs(sig / BO.surface_tension(A_BIN, B_BIN, K_BIN) - 1) < 1e-10


def _drop_state(m, n=32, R=8.0, perturb=1e-3, seed=7, sign=1.0):
    shape = (1, n, n)
    w = BO.interface_width(m.A, m.kappa)
    phi0 = sign * BO.drop_phi(shape, [(n / 2, n / 2)], [R], 1.0, -1.0, w)
    rho0 = 1.0 + perturb * inputs.noise(seed, shape)
    return BO.init_equilibrium(rho0, phi0, m)


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_conservation(scheme):
    """Mass, total order parameter and momentum are conserved to rounding."""
    m = _model(scheme, tau=0.8, tau_phi=0.9)
    f, g = _drop_state(m)
    d0 = BO.diagnostics(f, g, m)
    f, g = BO.run(f, g, m, 60)
    d1 = BO.diagnostics(f, g, m)
    assert abs(d1["mass"] - d0["mass"]) < 1e-10
    assert abs(d1["phi_total"] - d0["phi_total"]) < 1e-10
    for a in range(2):
        assert abs(d1["momentum"][a] - d0["momentum"][a]) < 1e-11
    assert d1["max_u"] > 0   # the drop does move


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_phi_sign_symmetry(scheme):
    """psi is even in phi (B1): the state from -phi0 is -phi with the same rho and u."""
    m = _model(scheme)
    fa, ga = _drop_state(m, sign=1.0)
    fb, gb = _drop_state(m, sign=-1.0)
    fa, ga = BO.run(fa, ga, m, 40)
    fb, gb = BO.run(fb, gb, m, 40)
    assert np.abs(fa - fb).max() < 1e-13
    assert np.abs(ga + gb).max() < 1e-13


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_uniform_bulk_is_a_fixed_point(scheme):
    """A uniform bulk phase at rest is left unchanged."""
    m = _model(scheme)
    shape = (1, 6, 7)
    f, g = BO.init_equilibrium(np.full(shape, 1.1), np.full(shape, -BO.phi_star(A_BIN, B_BIN)), m)
    f1, g1 = BO.run(f, g, m, 5)
    assert np.abs(f1 - f).max() < 1e-15 and np.abs(g1 - g).max() < 1e-15   # rounding only


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_flat_interface_stays_near_tanh_profile(scheme):
    """Two flat interfaces phi* tanh(+-(x - x_k)/w): after 800 steps the profile is
    within 2% of phi* of the continuum one (the lattice Laplacian's error at w = 2
    sites), the flow has decayed below 1e-5 and mu (zero in the continuum) below
    1e-4."""
    m = _model(scheme)
    nx, ny = 64, 4
    x = np.arange(nx, dtype=np.float64)[None, None, :] * np.ones((1, ny, 1))
    w = BO.interface_width(A_BIN, K_BIN)
    phi0 = np.tanh((x - 16) / w) - np.tanh((x - 48) / w) - 1.0
    f, g = BO.init_equilibrium(np.ones_like(phi0), phi0, m)
    f, g = BO.run(f, g, m, 800)
    rho, phi, u, v, mu = BO.observables(f, g, m)
    assert np.abs(phi - phi0).max() < 0.02
    assert max(np.abs(v[0]).max(), np.abs(v[1]).max()) < 1e-5
    assert np.abs(mu).max() < 1e-4
    assert np.abs(phi - phi[:, :1, :]).max() < 1e-12     # stays uniform in y


def _laplace(scheme, n, R, steps):
    m = _model(scheme)
    shape = (1, n, n)
    phi0 = BO.drop_phi(shape, [(n / 2, n / 2)], [R], 1.0, -1.0, BO.interface_width(A_BIN, K_BIN))
    f, g = BO.run(*BO.init_equilibrium(np.ones(shape), phi0, m), m, steps)
    rho, phi, u, v, _ = BO.observables(f, g, m)
    c = (0, n // 2, n // 2)
    pin, pout = phi[c], phi[0, 0, 0]
    R_e = np.sqrt((phi.sum() - pout * n * n) / (np.pi * (pin - pout)))   # equimolar radius
    dP = BO.p0(rho[c], pin, A_BIN, B_BIN) - BO.p0(rho[0, 0, 0], pout, A_BIN, B_BIN)
    return dP * R_e / BO.surface_tension(A_BIN, B_BIN, K_BIN), float(np.sqrt(v[0] ** 2 + v[1] ** 2).max())


@pytest.mark.slow
def test_laplace_law_and_forcing_reduction():
    """dP R / sigma = 1 within the interface discretisation (w = 2 sites) in both
    schemes, and the forcing scheme's max|v| is well below the equilibrium scheme's."""
    eq, v_eq = _laplace("equilibrium", 48, 10.0, 2000)
    fo, v_fo = _laplace("forcing", 48, 10.0, 2000)
    assert abs(eq - 1) < 0.06, eq
    assert abs(fo - 1) < 0.06, fo
    assert v_fo < v_eq / 2.5, (v_fo, v_eq)


def _mode_amplitude(field_1d, k):
    n = field_1d.size
    return float((field_1d * np.sin(k * np.arange(n))).sum() * 2 / n)


@pytest.mark.parametrize("tau_phi", [0.8, 1.3])
def test_order_parameter_diffuses_with_mobility(tau_phi):
    """B = kappa = 0, A > 0: mu = A phi and the phi equation is diffusion with
    D = Gamma A (tau_phi - 1/2) (mobility Gamma (tau_phi - 1/2), B6); a sine mode
    decays as exp(-D k^2 t) (1% for k = 2 pi / 64 over 300 steps)."""
    n, t = 64, 300
    k = 2 * np.pi / n
    m = BO.BinaryModel("D2Q9", 0.3, 0.0, 0.0, 0.5, 1.2, tau_phi)
    x = np.arange(n)[None, None, :] * np.ones((1, 4, 1))
    phi0 = 1e-3 * np.sin(k * x)
    f, g = BO.run(*BO.init_equilibrium(np.ones_like(phi0), phi0, m), m, t)
    phi = BO.observables(f, g, m)[1]
    D = m.Gamma * m.A * (tau_phi - 0.5)
    assert abs(_mode_amplitude(phi[0, 0], k) / 1e-3 / np.exp(-D * k * k * t) - 1) < 0.01


@pytest.mark.parametrize("tau", [0.7, 1.4])
def test_shear_wave_decays_with_viscosity(tau):
    """In a bulk phase a shear wave u_x = U sin(k y) decays as exp(-nu k^2 t),
    nu = (tau - 1/2)/3 (the BGK viscosity of Eq. 4; 1% for k = 2 pi / 64)."""
    n, t = 64, 300
    k = 2 * np.pi / n
    m = _model(tau=tau)
    y = np.arange(n)[None, :, None] * np.ones((1, 1, 4))
    ux = 1e-4 * np.sin(k * y)
    f, g = BO.init_equilibrium(np.ones_like(ux), np.ones_like(ux), m, u0=[ux, np.zeros_like(ux)])
    f, g = BO.run(f, g, m, t)
    u = BO.observables(f, g, m)[2]
    nu = (tau - 0.5) / 3
    assert abs(_mode_amplitude(u[0][0, :, 0], k) / 1e-4 / np.exp(-nu * k * k * t) - 1) < 0.01


# ---------------------------------------------------------------- D3Q19 (Sec. VII weights)

def _smooth_fields_3d(n=(12, 10, 8), seed=5):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = inputs.noise(seed, (8,))
    kx, ky, kz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    rho = 1.0 + 0.05 * np.sin(kx * x + r[0]) * np.cos(kz * z + r[1])
    phi = 0.8 * np.sin(kx * x + r[2]) + 0.1 * np.cos(ky * y + r[3]) + 0.05 * np.sin(kz * z + r[4])
    u = [0.03 * np.cos(ky * y + r[5]), 0.02 * np.sin(kz * z + r[6]), 0.01 * np.cos(kx * x + r[7])]
    return rho, phi, u


def _model3(scheme="equilibrium", **kw):
    p = dict(A=A_BIN, B=B_BIN, kappa=K_BIN, Gamma=0.7, tau=0.8, tau_phi=0.9)
    p.update(kw)
    return BO.BinaryModel("D3Q19", p["A"], p["B"], p["kappa"], p["Gamma"], p["tau"], p["tau_phi"], scheme=scheme)


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_f_and_g_moments_d3q19(scheme):
    """The D3Q19 weights (Eq. 31 with readings R4, R5) give the moments of B3 / B5 in 3D."""
    m = _model3(scheme)
    rho, phi, u = _smooth_fields_3d()
    grad = O.gradient(phi, m.stencils)
    lap = O.laplacian(phi, m.stencils)
    feq = BO.equilibrium_f(rho, phi, u, grad, lap, m, include_m_terms=scheme == "equilibrium")
    mu = m.A * phi + m.B * phi ** 3 - m.kappa * lap
    geq = BO.equilibrium_g(phi, u, BO.chemical_potential(phi, lap, m.A, m.B, m.kappa), m)
    e = m.e.astype(np.float64)
    g2 = sum(ga ** 2 for ga in grad)
    assert np.abs(feq.sum(axis=0) - rho).max() < 1e-15 and np.abs(geq.sum(axis=0) - phi).max() < 1e-15
    for a in range(3):
        assert np.abs(np.einsum("i,i...->...", e[:, a], feq) - rho * u[a]).max() < 1e-15
        assert np.abs(np.einsum("i,i...->...", e[:, a], geq) - phi * u[a]).max() < 1e-15
        for b in range(3):
            P = (BO.p0(rho, phi, m.A, m.B) - m.kappa * phi * lap - 0.5 * m.kappa * g2) * (a == b) \
                + m.kappa * grad[a] * grad[b]
            if scheme == "forcing":
                P = P - m.kappa * (grad[a] * grad[b] - 0.5 * g2 * (a == b))
            mf = np.einsum("i,i,i...->...", e[:, a], e[:, b], feq)
            mg = np.einsum("i,i,i...->...", e[:, a], e[:, b], geq)
            assert np.abs(mf - (P + rho * u[a] * u[b])).max() < 1e-14, (a, b)
            assert np.abs(mg - (m.Gamma * mu * (a == b) + phi * u[a] * u[b])).max() < 1e-15, (a, b)


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_conservation_and_symmetry_d3q19(scheme):
    """3D: mass, sum phi and momentum conserved; phi -> -phi symmetric; uniform bulk fixed."""
    m = _model3(scheme)
    shape = (10, 12, 14)
    w = BO.interface_width(m.A, m.kappa)
    phi0 = BO.drop_phi(shape, [(7.0, 6.0, 5.0)], [4.0], 1.0, -1.0, w)
    rho0 = 1.0 + 1e-3 * inputs.noise(9, shape)
    out = []
    for sign in (1.0, -1.0):
        f, g = BO.init_equilibrium(rho0, sign * phi0, m)
        d0 = BO.diagnostics(f, g, m)
        f, g = BO.run(f, g, m, 25)
        d1 = BO.diagnostics(f, g, m)
        assert abs(d1["mass"] - d0["mass"]) < 1e-10 and abs(d1["phi_total"] - d0["phi_total"]) < 1e-10
        for a in range(3):
            assert abs(d1["momentum"][a] - d0["momentum"][a]) < 1e-11
        out.append((f, g))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-13 and np.abs(out[0][1] + out[1][1]).max() < 1e-13
    fb, gb = BO.init_equilibrium(np.full((3, 4, 5), 1.2), np.full((3, 4, 5), 1.0), m)
    f1, g1 = BO.run(fb, gb, m, 3)
    assert np.abs(f1 - fb).max() < 1e-15 and np.abs(g1 - gb).max() < 1e-15


def test_shear_wave_d3q19():
    """A shear wave u_x = U sin(k z) in a bulk phase decays as exp(-nu k^2 t), nu = (tau - 1/2)/3."""
    n, t, tau = 32, 150, 1.1
    k = 2 * np.pi / n
    m = _model3(tau=tau)
    z = np.arange(n)[:, None, None] * np.ones((1, 2, 2))
    ux = 1e-4 * np.sin(k * z)
    f, g = BO.init_equilibrium(np.ones_like(ux), np.ones_like(ux), m, u0=[ux, 0 * ux, 0 * ux])
    f, g = BO.run(f, g, m, t)
    u = BO.observables(f, g, m)[2]
    nu = (tau - 0.5) / 3
    assert abs(_mode_amplitude(u[0][:, 0, 0], k) / 1e-4 / np.exp(-nu * k * k * t) - 1) < 0.01


def thermodynamic_residual(p0_fn=None, mu_fn=None, n=256):
    """Relative residual of d_x P_xx = phi d_x mu (B2, B3 at uniform rho; the
    Gibbs-Duhem relation of the free energy B1) on a long-wavelength phi(x),
    with the discrete gradient and Laplacian of B8 and spectral d_x."""
    p0_fn = p0_fn or BO.p0
    mu_fn = mu_fn or BO.chemical_potential
    m = _model()
    x = np.arange(n, dtype=np.float64)
    phi = (0.8 * np.sin(2 * np.pi * x / n) + 0.3 * np.cos(4 * np.pi * x / n))[None, None, :] * np.ones((1, 4, 1))
    rho = np.ones_like(phi)
    grad = O.gradient(phi, m.stencils)
    lap = O.laplacian(phi, m.stencils)
    g2 = grad[0] ** 2 + grad[1] ** 2
    pxx = p0_fn(rho, phi, m.A, m.B) - m.kappa * phi * lap - 0.5 * m.kappa * g2 + m.kappa * grad[0] ** 2
    mu = mu_fn(phi, lap, m.A, m.B, m.kappa)
    k = 2j * np.pi * np.fft.fftfreq(n)
    ddx = lambda a: np.real(np.fft.ifft(k * np.fft.fft(a[0, 0])))
    lhs, rhs = ddx(pxx), phi[0, 0] * ddx(mu)
    return float(np.abs(lhs - rhs).max() / np.abs(rhs).max())


def test_pressure_tensor_is_thermodynamically_consistent():
    """d_b P_ab = phi d_a mu at uniform rho (Gibbs-Duhem of B1): the p0 of B2 and the
    tensor of B3 belong to the chemical potential of B2 (residual 5e-7 at wavelengths of
    128 and 256 sites; bound 1e-5 - a wrong p0 or a wrong sign of the gradient term of mu
    leave 0.6 and 4e-3)."""
    assert thermodynamic_residual() < 1e-5
