"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

float64 storage: element-by-element agreement of every population, to the
1e-12 relative bound, after up to 1000 steps, on ragged grids that span
several CTA tiles.  Reduced storage: stated tolerances (see the test bodies).
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from paper_0710_5470_gb300 import inputs
from tests.helpers import drop_populations, library, make_ctx, oracle_model, rel_inf

pytestmark = pytest.mark.gpu

F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3

# odd nx: one site per halo load; even nx: two (32-bit arithmetic paths)
CASES = [
    ("D2Q9", "equilibrium", (45, 37)),
    ("D2Q9", "forcing", (45, 37)),
    ("D2Q9", "equilibrium", (46, 37)),
    ("D2Q9", "forcing", (46, 37)),
    ("D3Q19", "equilibrium", (37, 13, 11)),
    ("D3Q19", "forcing", (37, 13, 11)),
    ("D3Q19", "equilibrium", (38, 13, 11)),
    ("D3Q19", "forcing", (38, 13, 11)),
]


@pytest.mark.parametrize("lat,scheme,shape", CASES)
def test_f64_step_parity_ragged(lat, scheme, shape):
    """50 steps from a perturbed drop: every f_i within 1e-12 of the oracle."""
    lb = library()
    m = oracle_model(lat, scheme)
    R = 0.3 * min(shape)
    f0 = drop_populations(m, shape, R, perturb=1e-3, seed=3)
    with make_ctx(lb, lat, scheme, shape) as ctx:
        ctx.set_populations(f0)
        assert np.array_equal(ctx.get_populations(), f0)
        ctx.step(50)
        got = ctx.get_populations()
    want = O.run(f0, m, 50)
    for i in range(len(f0)):
        assert rel_inf(got[i], want[i]) < 1e-12, (i, rel_inf(got[i], want[i]))


@pytest.mark.parametrize("lat,scheme,shape", [
    ("D2Q9", "equilibrium", (40, 36)), ("D2Q9", "forcing", (40, 36)),
    ("D3Q19", "equilibrium", (22, 20, 18)), ("D3Q19", "forcing", (22, 20, 18))])
def test_f64_parity_1000_steps(lat, scheme, shape):
    """1e-12 relative per field after 1000 steps: every f_i and rho relative to
    their maximum; u and v relative to max(|u|, 1e-3 c).  u = j/rho with j a
    sum of O(1) populations, so its rounding floor is ~eps*rho ~ 1e-16
    absolute; the 1e-3 c floor keeps the bound (1e-15) above it."""
    lb = library()
    m = oracle_model(lat, scheme, tau=1.0)
    f0 = drop_populations(m, shape, 0.3 * min(shape))
    with make_ctx(lb, lat, scheme, shape, tau=1.0) as ctx:
        ctx.set_populations(f0)
        ctx.step(1000)
        got = ctx.get_populations()
        rho_g, u_g, v_g = ctx.fields()
    want = O.run(f0, m, 1000)
    for i in range(len(f0)):
        assert rel_inf(got[i], want[i]) < 1e-12
    rho, u, v = O.observables(want, m)
    assert rel_inf(rho_g, rho) < 1e-12
    umax = max(max(np.abs(x).max() for x in u), 1e-3)
    assert max(np.abs(x).max() for x in u) > 1e-7       # the drop survived: u is not rounding noise
    for a in range(m.dim):
        assert np.abs(u_g[a] - u[a]).max() / umax < 1e-12
        assert np.abs(v_g[a] - v[a]).max() / umax < 1e-12


@pytest.mark.parametrize("lat,scheme", [("D2Q9", "equilibrium"), ("D2Q9", "forcing"),
                                        ("D3Q19", "equilibrium"), ("D3Q19", "forcing")])
def test_init_drops_parity(lat, scheme):
    """lb_init_drops: tanh drops (two, one wrapping the boundary) then f^eq."""
    lb = library()
    m = oracle_model(lat, scheme)
    shape = (40, 34) if lat == "D2Q9" else (20, 18, 16)
    if lat == "D2Q9":
        centres, radii = [(20.0, 17.0), (2.0, 1.5)], [7.0, 5.0]
    else:
        centres, radii = [(10.0, 9.0, 8.0), (1.0, 17.0, 0.5)], [4.5, 3.0]
    with make_ctx(lb, lat, scheme, shape) as ctx:
        ctx.init_drops(centres, radii, width=2.0)
        got = ctx.get_populations()
        rl, rg = ctx.coexistence()
    nx, ny, nz = (tuple(shape) + (1,))[:3]
    orl, org = O.coexistence(m.a, m.b, m.T)
    assert abs(rl - orl) < 1e-12 * orl
    rho0 = O.drop_density((nz, ny, nx), centres, radii, orl, org, width=2.0)
    want = O.init_equilibrium(rho0, m)
    for i in range(len(want)):
        assert rel_inf(got[i], want[i]) < 1e-13


@pytest.mark.parametrize("lat,scheme", [("D2Q9", "forcing"), ("D3Q19", "forcing"), ("D3Q19", "equilibrium")])
def test_fields_and_stats_parity(lat, scheme):
    """lb_fields (rho, u, v of Eq. 40) and lb_stats_get against the oracle."""
    lb = library()
    m = oracle_model(lat, scheme)
    shape = (33, 30) if lat == "D2Q9" else (17, 14, 12)
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-4, seed=5)
    with make_ctx(lb, lat, scheme, shape) as ctx:
        ctx.set_populations(f0)
        ctx.step(20)
        rho_g, u_g, v_g = ctx.fields()
        st = ctx.stats()
    f = O.run(f0, m, 20)
    rho, u, v = O.observables(f, m)
    d = O.diagnostics(f, m)
    assert rel_inf(rho_g, rho) < 1e-13
    for a in range(m.dim):
        assert np.abs(u_g[a] - u[a]).max() < 1e-13
        assert np.abs(v_g[a] - v[a]).max() < 1e-13
    assert abs(st["mass"] - d["mass"]) < 1e-12 * d["mass"]
    for a in range(m.dim):
        assert abs(st["momentum"][a] - d["momentum"][a]) < 1e-12 * d["mass"]
    assert abs(st["max_u"] - d["max_u"]) < 1e-12
    assert abs(st["max_v"] - d["max_v"]) < 1e-12
    assert st["step"] == 20 and st["status"] == 0


@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 1)), ("D2Q9", (1, 7)), ("D2Q9", (5, 2)),
                                       ("D3Q19", (1, 1, 1)), ("D3Q19", (3, 1, 2)), ("D3Q19", (2, 5, 1))])
@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_degenerate_tiny_grids(lat, shape, scheme):
    """Grids narrower than the stencil wrap onto themselves; still exact."""
    lb = library()
    m = oracle_model(lat, scheme)
    nx, ny, nz = (tuple(shape) + (1,))[:3]
    rng_f = drop_populations(m, shape, 1.0)
    f0 = rng_f * (1.0 + 1e-2 * inputs.noise(11, rng_f.shape))
    with make_ctx(lb, lat, scheme, shape) as ctx:
        ctx.set_populations(f0)
        ctx.step(7)
        got = ctx.get_populations()
    want = O.run(f0, m, 7)
    assert rel_inf(got, want) < 1e-12


@pytest.mark.parametrize("storage,tol", [(F32, 1e-5), (F16DEV, 5e-4), (BF16DEV, 5e-3)])
@pytest.mark.parametrize("lat,shape", [("D2Q9", (1, 7)), ("D2Q9", (2, 5)), ("D3Q19", (1, 1, 1)),
                                       ("D3Q19", (2, 5, 1)), ("D3Q19", (2, 2, 3))])
@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_degenerate_tiny_grids_reduced_storage(lat, shape, scheme, storage, tol):
    """The same wrap-onto-itself grids in reduced storage (nx = 2 takes the
    paired halo loads), from the rounded start, within the storage's bound."""
    lb = library()
    m = oracle_model(lat, scheme)
    rng_f = drop_populations(m, shape, 1.0)
    f0 = rng_f * (1.0 + 1e-2 * inputs.noise(12, rng_f.shape))
    with make_ctx(lb, lat, scheme, shape, storage=storage) as ctx:
        ctx.set_populations(f0)
        start = ctx.get_populations()
        ctx.step(7)
        got = ctx.get_populations()
    want = O.run(start, m, 7)
    assert rel_inf(got, want) < tol


def test_zero_steps_and_state_errors():
    lb = library()
    with make_ctx(lb, "D2Q9", "forcing", (16, 16)) as ctx:
        with pytest.raises(lb.LBError) as e:
            ctx.step(1)                     # step before init
        assert e.value.status == 6
        ctx.init_drops([(8.0, 8.0)], [4.0])
        f = ctx.get_populations()
        ctx.step(0)
        assert np.array_equal(ctx.get_populations(), f)
        with pytest.raises(lb.LBError):
            ctx.step(-1)


def test_nonfinite_density_is_reported_and_sticky():
    """A NaN planted in the host state raises LB_EUNSTABLE at the next sync,
    and the context keeps returning it (no GPU fault involved)."""
    lb = library()
    m = oracle_model("D2Q9", "equilibrium")
    f0 = drop_populations(m, (16, 16), 4.0)
    f0[0, 0, 3, 3] = np.nan
    with make_ctx(lb, "D2Q9", "equilibrium", (16, 16)) as ctx:
        ctx.set_populations(f0)
        ctx.step(2)
        with pytest.raises(lb.LBError) as e:
            ctx.synchronize()
        assert e.value.status == 4
        with pytest.raises(lb.LBError) as e:
            ctx.step(1)
        assert e.value.status == 4


# ------------------------------------------------------------ reduced storage

def _reduced_case(lat, scheme, storage, shape, steps):
    lb = library()
    m = oracle_model(lat, scheme)
    f0 = drop_populations(m, shape, 0.3 * min(shape))
    with make_ctx(lb, lat, scheme, shape, storage=storage) as ctx:
        ctx.set_populations(f0)
        start = ctx.get_populations()          # f0 rounded to the storage
        ctx.step(steps)
        got = ctx.get_populations()
        rho_g, u_g, v_g = ctx.fields()
    want = O.run(start, m, steps)
    rho, u, v = O.observables(want, m)
    return got, want, rho_g, rho, v_g, v


@pytest.mark.parametrize("lat,scheme,shape", CASES)
def test_f32_storage_tolerance(lat, scheme, shape):
    """float32 storage and arithmetic, 100 steps: rho within 1e-5 relative,
    populations within 2e-5 of max|f|, v within 1e-6 absolute."""
    got, want, rho_g, rho, v_g, v = _reduced_case(lat, scheme, F32, shape, 100)
    assert rel_inf(rho_g, rho) < 1e-5
    assert rel_inf(got, want) < 2e-5
    assert max(np.abs(v_g[a] - v[a]).max() for a in range(len(v))) < 1e-6


@pytest.mark.parametrize("storage,tol_rho,tol_v", [(F16DEV, 3e-5, 1e-5), (BF16DEV, 2e-4, 6e-5)])
@pytest.mark.parametrize("lat,scheme,shape", CASES)
def test_deviation_storage_tolerance(lat, scheme, shape, storage, tol_rho, tol_v):
    """fp16 / bf16 deviation storage (f_0 float32), 100 steps from the rounded
    start: rho within tol_rho relative, v within tol_v absolute.  Each step
    rounds every deviation to the format (11 / 8 significant bits); measured
    maxima over these cases on GB300: fp16 rho 1.3e-5, v 3.1e-6; bf16 rho
    7.8e-5, v 2.5e-5; the bounds leave a factor ~2.5."""
    got, want, rho_g, rho, v_g, v = _reduced_case(lat, scheme, storage, shape, 100)
    assert rel_inf(rho_g, rho) < tol_rho
    assert max(np.abs(v_g[a] - v[a]).max() for a in range(len(v))) < tol_v


@pytest.mark.parametrize("storage", [F32, F16DEV, BF16DEV])
@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
@pytest.mark.parametrize("shape", [(66, 20, 9), (2, 5, 3)])
def test_paired_halo_loads_are_bit_identical(storage, scheme, shape, monkeypatch):
    """With an even nx the tile kernel's halo stage loads two adjacent sites
    per access; it must give exactly the one-site form's result (same
    arithmetic, same order), over ragged tiles and a lattice narrower than one
    pair of halo columns.  (LB_D3_VARIANT=0 selects the tile kernel for both
    schemes, whose default with 32-bit arithmetic storage is the pair kernel,
    checked against the oracle in test_pair_kernel_parity.)"""
    monkeypatch.setenv("LB_D3_VARIANT", "0")
    lb = library()
    m = oracle_model("D3Q19", scheme)
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=9)
    outs = []
    for no_pair in (False, True):
        if no_pair:
            monkeypatch.setenv("LB_NO_PAIR", "1")
        else:
            monkeypatch.delenv("LB_NO_PAIR", raising=False)
        with make_ctx(lb, "D3Q19", scheme, shape, storage=storage) as ctx:
            ctx.set_populations(f0)
            ctx.step(25)
            outs.append(ctx.get_populations())
    assert np.isfinite(outs[0]).all()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("kernel", ["pairs", "tile"])
@pytest.mark.parametrize("storage", [F32, F16DEV, BF16DEV])
@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
@pytest.mark.parametrize("shape", [(66, 20), (2, 5), (34, 47)])
def test_paired_halo_loads_are_bit_identical_2d(storage, scheme, shape, kernel, monkeypatch):
    """The D2Q9 step with an even nx moves two sites per access (the pair
    kernel everywhere, the tile kernel in its halo stage); it gives exactly
    the result of the same kernel moving one site per access."""
    monkeypatch.setenv("LB_D2_VARIANT", "1" if kernel == "pairs" else "0")
    lb = library()
    m = oracle_model("D2Q9", scheme)
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=8)
    outs = []
    for no_pair in (False, True):
        if no_pair:
            monkeypatch.setenv("LB_NO_PAIR", "1")
        else:
            monkeypatch.delenv("LB_NO_PAIR", raising=False)
        with make_ctx(lb, "D2Q9", scheme, shape, storage=storage) as ctx:
            ctx.set_populations(f0)
            ctx.step(25)
            outs.append(ctx.get_populations())
    assert np.isfinite(outs[0]).all()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("storage,tol_f,tol_rho", [(F16DEV, 1e-5, 1e-5), (BF16DEV, 8e-5, 6e-5), (F32, 2e-6, 2e-6)])
@pytest.mark.parametrize("variant", ["default", "1", "2", "4", "8", "9", "10", "14", "15", "16", "25"])
@pytest.mark.parametrize("shape", [(68, 20, 12), (2, 3, 3), (130, 10, 40), (64, 16, 9), (96, 20, 7), (32, 5, 3)])
def test_pair_kernel_parity(shape, variant, storage, tol_f, tol_rho, monkeypatch):
    """The D3Q19 forcing-scheme pair kernel (two x sites per thread, packed
    float32 pairs) in every tile / prefetch form, one and five steps from the
    same rounded state as the oracle: every population within tol_f of
    max|f| and rho within tol_rho relative (one rounding of the collided
    deviations to the format per step; ragged tiles in x and y, a lattice
    narrower than one pair of halo columns, several z chunks).  With 16-bit
    storage and nx a multiple of 32 (64, 96, 32 here) the populations are in
    the interleaved block layout, which the import / export kernels share."""
    if variant == "default":
        monkeypatch.delenv("LB_D3_VARIANT", raising=False)
    else:
        monkeypatch.setenv("LB_D3_VARIANT", variant)
    lb = library()
    m = oracle_model("D3Q19", "forcing")
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=5)
    for steps in (1, 5):
        with make_ctx(lb, "D3Q19", "forcing", shape, storage=storage) as ctx:
            ctx.set_populations(f0)
            start = ctx.get_populations()
            ctx.step(steps)
            got = ctx.get_populations()
            rho_g, _, _ = ctx.fields(want_v=False)
            form = ctx.kernel_info()["form"]
        if storage != F32 or variant != "default":
            assert form.startswith("pairs"), form
        want = O.run(start, m, steps)
        rho = want.sum(axis=0)
        assert rel_inf(got, want) < tol_f * steps, (steps, rel_inf(got, want))
        assert rel_inf(rho_g, rho) < tol_rho * steps



@pytest.mark.parametrize("storage,tol_f", [(F32, 2e-6), (F16DEV, 1e-5), (BF16DEV, 8e-5)])
@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
@pytest.mark.parametrize("shape", [(45, 37), (46, 37), (64, 16), (3, 9), (2, 2), (130, 7)])
def test_d2q9_pair_and_tile_kernels(shape, scheme, storage, tol_f, monkeypatch):
    """The D2Q9 pair kernel (two x sites per thread, packed float32 pairs;
    odd nx: every site loaded and stored on its own) and the one-site tile
    kernel, one and five steps from the same rounded state as the oracle:
    every population within tol_f of max|f| per step."""
    lb = library()
    m = oracle_model("D2Q9", scheme)
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=9)
    for variant, form in (("1", "pairs"), ("0", "tile")):
        monkeypatch.setenv("LB_D2_VARIANT", variant)
        for steps in (1, 5):
            with make_ctx(lb, "D2Q9", scheme, shape, storage=storage) as ctx:
                ctx.set_populations(f0)
                start = ctx.get_populations()
                ctx.step(steps)
                got = ctx.get_populations()
                assert ctx.kernel_info()["form"].startswith(form)
            want = O.run(start, m, steps)
            assert rel_inf(got, want) < tol_f * steps, (variant, steps, rel_inf(got, want))


@pytest.mark.parametrize("storage,tol_f,tol_rho", [(F16DEV, 1e-5, 1e-5), (BF16DEV, 8e-5, 6e-5), (F32, 2e-6, 2e-6)])
@pytest.mark.parametrize("shape", [(68, 20, 12), (2, 3, 3), (130, 10, 40), (64, 16, 9), (96, 20, 7), (32, 5, 3),
                                   (64, 8, 1)])
def test_equilibrium_pair_kernel_parity(shape, storage, tol_f, tol_rho, monkeypatch):
    """The D3Q19 equilibrium-scheme pair kernel (two x sites per thread, packed
    float32 pairs, the M terms of the optimal weights in the collision; the
    interleaved 16-bit layout when nx is a multiple of 32), one and five steps
    from the same rounded state as the oracle."""
    monkeypatch.delenv("LB_D3_VARIANT", raising=False)
    lb = library()
    m = oracle_model("D3Q19", "equilibrium")
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=7)
    for steps in (1, 5):
        with make_ctx(lb, "D3Q19", "equilibrium", shape, storage=storage) as ctx:
            ctx.set_populations(f0)
            start = ctx.get_populations()
            ctx.step(steps)
            got = ctx.get_populations()
            rho_g, _, _ = ctx.fields(want_v=False)
            assert ctx.kernel_info()["form"].startswith("pairs"), ctx.kernel_info()["form"]
        want = O.run(start, m, steps)
        rho = want.sum(axis=0)
        assert rel_inf(got, want) < tol_f * steps, (steps, rel_inf(got, want))
        assert rel_inf(rho_g, rho) < tol_rho * steps
