"""Binary-fluid kernels (csrc/binary2d.cu D2Q9, csrc/binary3d.cu D3Q19) against
the binary oracle.

float64: every population, rho, phi, u, v and mu to 1e-12 after 100 steps on
ragged, odd and tiny lattices, both schemes; the initial state to 1e-14; one
step at 1024^2.  float32 (two sites per thread for even nx): the same comparison
at float32 rounding, and one step at the bench's 2048^2.  fp16 deviations (D2Q9,
even nx): one and 20 steps against the oracle from the stored state, and
Laplace's law.  The graph
replay path equals single launches bit for bit; mass, order parameter and
momentum stay conserved; Laplace's law holds on the device.  D3Q19: the same
float64 parity after 30 steps, the initial state, float32, graph replay,
conservation, the 3D Laplace law and one step at 96^3.
"""
import numpy as np
import pytest

from oracle import binary_oracle as BO
from paper_0710_5470_gb300 import inputs
from tests.helpers import library, rel_inf

pytestmark = pytest.mark.gpu

A_BIN, B_BIN, K_BIN = -0.04, 0.04, 0.08     # phi* = 1, interface width w = 2
SCHEMES = ["equilibrium", "forcing"]


def _model(scheme, tau=0.8, tau_phi=0.9, Gamma=0.7):
    return BO.BinaryModel("D2Q9", A_BIN, B_BIN, K_BIN, Gamma, tau, tau_phi, scheme=scheme)


def _ctx(lb, m, shape_xy, storage=0):
    return lb.BinaryContext(shape_xy, m.A, m.B, m.kappa, m.Gamma, m.tau, m.tau_phi,
                            scheme=lb.FORCING if m.scheme == "forcing" else lb.EQUILIBRIUM, storage=storage)


def _fields(m, nx, ny, R=None, seed=1):
    """A drop of phase +phi* in -phi*, rho = 1 + 1e-3 noise, u = 1e-3 noise (seeded)."""
    shape = (1, ny, nx)
    R = R if R is not None else 0.3 * min(nx, ny)
    phi0 = BO.drop_phi(shape, [(nx / 2, ny / 2)], [R], 1.0, -1.0, BO.interface_width(m.A, m.kappa))
    rho0 = 1.0 + 1e-3 * inputs.noise(seed, shape)
    u0 = [1e-3 * inputs.noise(seed + 1, shape), 1e-3 * inputs.noise(seed + 2, shape)]
    return rho0, phi0, u0


SHAPES = [(48, 20), (37, 11), (5, 3), (64, 16)]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", SHAPES)
def test_f64_parity(scheme, shape):
    m = _model(scheme)
    nx, ny = shape
    rho0, phi0, u0 = _fields(m, nx, ny)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, shape) as c:
        c.set_populations(f[:, 0], g[:, 0])
        c.step(100)
        fg, gg = c.get_populations()
        rho, phi, u, v, mu = c.fields()
        st = c.stats()
    fo, go = BO.run(f, g, m, 100)
    assert rel_inf(fg, fo[:, 0]) < 1e-12
    assert rel_inf(gg, go[:, 0]) < 1e-12
    orho, ophi, ou, ov, omu = BO.observables(fo, go, m)
    assert np.abs(rho - orho[0]).max() < 1e-12 and np.abs(phi - ophi[0]).max() < 1e-12
    for a in range(2):
        assert np.abs(u[a] - ou[a][0]).max() < 1e-14
        assert np.abs(v[a] - ov[a][0]).max() < 1e-14
    assert np.abs(mu - omu[0]).max() < 1e-13
    d = BO.diagnostics(fo, go, m)
    assert abs(st["mass"] - d["mass"]) < 1e-10 and abs(st["phi_total"] - d["phi_total"]) < 1e-10
    assert abs(st["max_v"] - d["max_v"]) < 1e-14 and st["step"] == 100 and st["status"] == 0


@pytest.mark.parametrize("scheme", SCHEMES)
def test_init_fields_matches_oracle(scheme):
    m = _model(scheme)
    nx, ny = 40, 24
    rho0, phi0, u0 = _fields(m, nx, ny)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, (nx, ny)) as c:
        c.init_fields(rho0[0], phi0[0], np.stack([u0[0][0], u0[1][0]]))
        fg, gg = c.get_populations()
    assert rel_inf(fg, f[:, 0]) < 1e-14 and rel_inf(gg, g[:, 0]) < 1e-14


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", [(48, 20), (36, 10), (6, 3), (37, 11)])
def test_f32_parity(scheme, shape):
    """float32 storage and arithmetic: 20 steps within 2e-6 of max |f| (float32
    rounding of ~100 operations per population and step, accumulated).  Even nx
    runs the two-sites-per-thread kernel (a ragged tile at 36, pairs wrapping at
    6), odd nx the one-site kernel."""
    m = _model(scheme)
    nx, ny = shape
    rho0, phi0, u0 = _fields(m, nx, ny)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, (nx, ny), storage=1) as c:
        c.set_populations(f[:, 0], g[:, 0])
        c.step(20)
        fg, gg = c.get_populations()
    fo, go = BO.run(f, g, m, 20)
    ef, eg = rel_inf(fg, fo[:, 0]), rel_inf(gg, go[:, 0])
    print(f"binary f32 {scheme} {shape}: f {ef:.2e} g {eg:.2e}")
    assert ef < 2e-6 and eg < 2e-6


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", [(48, 20), (36, 10), (6, 3)])
def test_f16dev_parity(scheme, shape):
    """fp16 deviations (f_0, g_0 float32; f_i - w_i p0(bulk) and g_i in fp16): one step from
    the stored state against the oracle stepping it in float64 within 3e-5 of max |f|, and
    20 steps from the rounded start within 1e-4 (measured on GB300: 4e-6 - 8e-6 and at most
    1.0e-5; one rounding of the deviations, below 0.02 here, to 11 significant bits is at
    most 1e-5 absolute per step, 2.5e-5 of max |f|)."""
    m = _model(scheme)
    nx, ny = shape
    rho0, phi0, u0 = _fields(m, nx, ny)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, (nx, ny), storage=2) as c:
        c.set_populations(f[:, 0], g[:, 0])
        fs, gs = c.get_populations()
        c.step(1)
        f1, g1 = c.get_populations()
        c.step(19)
        f20, g20 = c.get_populations()
    fo, go = BO.step(fs[:, None], gs[:, None], m)
    e1 = max(rel_inf(f1, fo[:, 0]), rel_inf(g1, go[:, 0]))
    fo, go = BO.run(fs[:, None], gs[:, None], m, 20)
    e20 = max(rel_inf(f20, fo[:, 0]), rel_inf(g20, go[:, 0]))
    print(f"binary f16dev {scheme} {shape}: 1 step {e1:.2e}, 20 steps {e20:.2e}")
    assert e1 < 3e-5 and e20 < 1e-4


def test_f16dev_laplace_law():
    """Laplace's law and the forcing scheme's smaller spurious velocity hold with fp16 deviations."""
    lb = library()
    n, R = 96, 20.0
    res = {}
    for scheme in SCHEMES:
        m = _model(scheme, tau=1.0, tau_phi=1.0, Gamma=1.0)
        phi0 = BO.drop_phi((1, n, n), [(n / 2, n / 2)], [R], 1.0, -1.0, BO.interface_width(A_BIN, K_BIN))
        with _ctx(lb, m, (n, n), storage=2) as c:
            c.init_fields(np.ones((n, n)), phi0[0])
            c.step(20000)
            rho, phi, u, v, mu = c.fields()
            st = c.stats()
        pin, pout = phi[n // 2, n // 2], phi[0, 0]
        R_e = np.sqrt((phi.sum() - pout * n * n) / (np.pi * (pin - pout)))
        dP = BO.p0(rho[n // 2, n // 2], pin, A_BIN, B_BIN) - BO.p0(rho[0, 0], pout, A_BIN, B_BIN)
        res[scheme] = (dP * R_e / BO.surface_tension(A_BIN, B_BIN, K_BIN), float(np.hypot(v[0], v[1]).max()))
        assert st["status"] == 0
    print("binary f16dev Laplace", res)
    for scheme in SCHEMES:
        assert abs(res[scheme][0] - 1) < 0.06, (scheme, res)
    assert res["forcing"][1] < res["equilibrium"][1], res


@pytest.mark.parametrize("storage", [0, 1])
def test_graph_replay_equals_single_launches(storage):
    m = _model("forcing")
    nx, ny = 64, 24
    rho0, phi0, u0 = _fields(m, nx, ny)
    lb = library()
    out = []
    for chunks in ([130], [1] * 130):
        with _ctx(lb, m, (nx, ny), storage=storage) as c:
            c.init_fields(rho0[0], phi0[0])
            for k in chunks:
                c.step(k)
            out.append(c.get_populations())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("scheme", SCHEMES)
def test_conservation_on_device(scheme):
    m = _model(scheme)
    nx, ny = 64, 64
    rho0, phi0, u0 = _fields(m, nx, ny)
    with _ctx(library(), m, (nx, ny)) as c:
        c.init_fields(rho0[0], phi0[0], np.stack([u0[0][0], u0[1][0]]))
        s0 = c.stats()
        c.step(3000)
        s1 = c.stats()
    assert abs(s1["mass"] / s0["mass"] - 1) < 1e-12
    assert abs(s1["phi_total"] - s0["phi_total"]) < 1e-9
    for a in range(2):
        assert abs(s1["momentum"][a] - s0["momentum"][a]) < 1e-11
    assert s1["status"] == 0 and s1["step"] == 3000


@pytest.mark.parametrize("storage", [0, 1])
def test_laplace_law_on_device(storage):
    """dP R / sigma = 1 (sigma = 4 kappa phi*^2 / (3 w)) within 5% for a drop of
    radius 20 after 20000 steps, both schemes; the forcing scheme's max|v| is
    below half the equilibrium scheme's."""
    lb = library()
    n, R = 96, 20.0
    res = {}
    for scheme in SCHEMES:
        m = _model(scheme, tau=1.0, tau_phi=1.0, Gamma=1.0)
        shape = (1, n, n)
        phi0 = BO.drop_phi(shape, [(n / 2, n / 2)], [R], 1.0, -1.0, BO.interface_width(A_BIN, K_BIN))
        with _ctx(lb, m, (n, n), storage=storage) as c:
            c.init_fields(np.ones((n, n)), phi0[0])
            c.step(20000)
            rho, phi, u, v, mu = c.fields()
        pin, pout = phi[n // 2, n // 2], phi[0, 0]
        R_e = np.sqrt((phi.sum() - pout * n * n) / (np.pi * (pin - pout)))
        dP = BO.p0(rho[n // 2, n // 2], pin, A_BIN, B_BIN) - BO.p0(rho[0, 0], pout, A_BIN, B_BIN)
        res[scheme] = (dP * R_e / BO.surface_tension(A_BIN, B_BIN, K_BIN), float(np.hypot(v[0], v[1]).max()))
    print("binary Laplace", storage, res)
    for scheme in SCHEMES:
        assert abs(res[scheme][0] - 1) < 0.05, (scheme, res)
    assert res["forcing"][1] < 0.5 * res["equilibrium"][1], res


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n, storage, tol", [(1024, 0, 1e-14), (2048, 1, 1e-6)])
def test_one_step_at_full_size(scheme, n, storage, tol):
    """One step on large lattices, every population: float64 at 1024^2, and the
    bench's configuration (2048^2, one drop of radius 512, float32 storage: the
    two-sites-per-thread kernel) from the float32-rounded state, against the
    oracle stepping that state in float64 (one step of float32 rounding)."""
    m = _model(scheme, tau=1.0, tau_phi=1.0, Gamma=1.0)
    rho0, phi0, u0 = _fields(m, n, n, R=n / 4, seed=11)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, (n, n), storage=storage) as c:
        c.set_populations(f[:, 0], g[:, 0])
        f, g = c.get_populations()          # the state as stored
        c.step(1)
        fg, gg = c.get_populations()
    fo, go = BO.step(f[:, None], g[:, None], m)
    assert rel_inf(fg, fo[:, 0]) < tol and rel_inf(gg, go[:, 0]) < tol


# ---------------------------------------------------------------- D3Q19

def _model3(scheme, tau=0.8, tau_phi=0.9, Gamma=0.7):
    return BO.BinaryModel("D3Q19", A_BIN, B_BIN, K_BIN, Gamma, tau, tau_phi, scheme=scheme)


def _fields3(m, nx, ny, nz, R=None, seed=21):
    shape = (nz, ny, nx)
    R = R if R is not None else 0.3 * min(nx, ny, nz)
    phi0 = BO.drop_phi(shape, [(nx / 2, ny / 2, nz / 2)], [R], 1.0, -1.0, BO.interface_width(m.A, m.kappa))
    rho0 = 1.0 + 1e-3 * inputs.noise(seed, shape)
    u0 = [1e-3 * inputs.noise(seed + k, shape) for k in (1, 2, 3)]
    return rho0, phi0, u0


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", [(20, 12, 10), (17, 9, 7), (5, 3, 4), (40, 8, 6)])
def test_d3q19_f64_parity(scheme, shape):
    """D3Q19 float64: every population, rho, phi, u, v and mu against the oracle
    after 30 steps (ragged bricks of 32 x 4 x 2, odd and tiny lattices)."""
    m = _model3(scheme)
    nx, ny, nz = shape
    rho0, phi0, u0 = _fields3(m, nx, ny, nz)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, shape) as c:
        c.set_populations(f, g)
        c.step(30)
        fg, gg = c.get_populations()
        rho, phi, u, v, mu = c.fields()
        st = c.stats()
    fo, go = BO.run(f, g, m, 30)
    assert rel_inf(fg, fo) < 1e-12 and rel_inf(gg, go) < 1e-12
    orho, ophi, ou, ov, omu = BO.observables(fo, go, m)
    assert np.abs(rho - orho).max() < 1e-12 and np.abs(phi - ophi).max() < 1e-12
    for a in range(3):
        assert np.abs(u[a] - ou[a]).max() < 1e-14 and np.abs(v[a] - ov[a]).max() < 1e-14
    assert np.abs(mu - omu).max() < 1e-13
    d = BO.diagnostics(fo, go, m)
    assert abs(st["mass"] - d["mass"]) < 1e-10 and abs(st["phi_total"] - d["phi_total"]) < 1e-10
    assert all(abs(st["momentum"][a] - d["momentum"][a]) < 1e-12 for a in range(3))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_d3q19_init_and_f32(scheme):
    """D3Q19: the device initial state matches the oracle's to 1e-14; float32 storage
    follows the oracle for 20 steps within 2e-6 of max |f|."""
    m = _model3(scheme)
    shape = (24, 10, 8)
    rho0, phi0, u0 = _fields3(m, *shape)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, shape) as c:
        c.init_fields(rho0, phi0, np.stack(u0))
        fg, gg = c.get_populations()
    assert rel_inf(fg, f) < 1e-14 and rel_inf(gg, g) < 1e-14
    with _ctx(library(), m, shape, storage=1) as c:
        c.set_populations(f, g)
        c.step(20)
        fg, gg = c.get_populations()
    fo, go = BO.run(f, g, m, 20)
    ef, eg = rel_inf(fg, fo), rel_inf(gg, go)
    print(f"binary D3Q19 f32 {scheme}: f {ef:.2e} g {eg:.2e}")
    assert ef < 2e-6 and eg < 2e-6


@pytest.mark.parametrize("storage", [0, 1])
def test_d3q19_graph_replay_and_conservation(storage):
    """Graph replay (two launches per step) equals single launches bit for bit;
    mass, sum phi and momentum stay conserved over 1000 steps."""
    m = _model3("forcing", tau=1.0, tau_phi=1.0, Gamma=1.0)
    shape = (32, 16, 12)
    rho0, phi0, u0 = _fields3(m, *shape, R=5.0)
    lb = library()
    out = []
    for chunks in ([130], [1] * 130):
        with _ctx(lb, m, shape, storage=storage) as c:
            c.init_fields(rho0, phi0)
            for k in chunks:
                c.step(k)
            out.append(c.get_populations())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    if storage == 0:
        with _ctx(lb, m, shape) as c:
            c.init_fields(rho0, phi0, np.stack(u0))
            s0 = c.stats()
            c.step(1000)
            s1 = c.stats()
        assert abs(s1["mass"] / s0["mass"] - 1) < 1e-12 and abs(s1["phi_total"] - s0["phi_total"]) < 1e-9
        assert all(abs(s1["momentum"][a] - s0["momentum"][a]) < 1e-11 for a in range(3))


@pytest.mark.parametrize("storage", [0, 1])
def test_d3q19_laplace_law(storage):
    """3D Laplace's law dP = 2 sigma / R (sigma = 4 kappa phi*^2 / (3 w)) within 6%
    for a drop of radius 12 in 48^3 after 8000 steps, both schemes; the forcing
    scheme's max|v| below the equilibrium scheme's."""
    lb = library()
    n, R = 48, 12.0
    res = {}
    for scheme in SCHEMES:
        m = _model3(scheme, tau=1.0, tau_phi=1.0, Gamma=1.0)
        shape = (n, n, n)
        phi0 = BO.drop_phi(shape, [(n / 2,) * 3], [R], 1.0, -1.0, BO.interface_width(A_BIN, K_BIN))
        with _ctx(lb, m, shape, storage=storage) as c:
            c.init_fields(np.ones(shape), phi0)
            c.step(8000)
            rho, phi, u, v, mu = c.fields()
        cen = (n // 2,) * 3
        pin, pout = phi[cen], phi[0, 0, 0]
        R_e = (3 * (phi.sum() - pout * n ** 3) / (4 * np.pi * (pin - pout))) ** (1 / 3)
        dP = BO.p0(rho[cen], pin, A_BIN, B_BIN) - BO.p0(rho[0, 0, 0], pout, A_BIN, B_BIN)
        res[scheme] = (dP * R_e / (2 * BO.surface_tension(A_BIN, B_BIN, K_BIN)),
                       float(np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2).max()))
    print("binary D3Q19 Laplace", storage, res)
    for scheme in SCHEMES:
        assert abs(res[scheme][0] - 1) < 0.06, (scheme, res)
    assert res["forcing"][1] < res["equilibrium"][1], res


@pytest.mark.parametrize("scheme", SCHEMES)
def test_d3q19_one_step_at_96(scheme):
    """One float64 step on 96^3 (a drop of radius 24), every population."""
    m = _model3(scheme, tau=1.0, tau_phi=1.0, Gamma=1.0)
    n = 96
    rho0, phi0, u0 = _fields3(m, n, n, n, R=24.0)
    f, g = BO.init_equilibrium(rho0, phi0, m, u0)
    with _ctx(library(), m, (n, n, n)) as c:
        c.set_populations(f, g)
        c.step(1)
        fg, gg = c.get_populations()
    fo, go = BO.step(f, g, m)
    assert rel_inf(fg, fo) < 1e-14 and rel_inf(gg, go) < 1e-14
