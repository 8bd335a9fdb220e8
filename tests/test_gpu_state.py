"""Checkpoint / restart (lb_get_state / lb_set_state) and the lb_stats
diagnostics dP and max_du against the oracle.

A run of N steps, exported, imported into a fresh context and continued for
N more steps must equal 2N steps of one context bit for bit, in every storage
format and population layout, including the step counter."""
import numpy as np
import pytest

from oracle import lb_oracle as O
from tests.helpers import drop_populations, library, make_ctx, oracle_model

pytestmark = pytest.mark.gpu

F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3


@pytest.mark.parametrize("storage", [F64, F32, F16DEV, BF16DEV])
@pytest.mark.parametrize("lat,scheme,shape", [
    ("D3Q19", "forcing", (64, 20, 12)),     # interleaved 16-bit layout (nx a multiple of 32)
    ("D3Q19", "forcing", (38, 13, 11)),     # one array per population
    ("D3Q19", "equilibrium", (38, 13, 11)),
    ("D3Q19", "equilibrium", (64, 16, 9)),  # the equilibrium pair kernel, interleaved 16-bit layout
    ("D2Q9", "forcing", (46, 37)),
    ("D2Q9", "equilibrium", (45, 37)),      # odd nx: the pair kernel site by site
])
def test_restart_is_bit_exact(lat, scheme, shape, storage):
    lb = library()
    m = oracle_model(lat, scheme)
    f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=4)
    n = 37
    with make_ctx(lb, lat, scheme, shape, storage=storage) as a:
        a.set_populations(f0)
        a.step(n)
        state = a.get_state()
        assert state[:8] == b"LBGBSTA1"
        a.step(n)
        want = a.get_state()
        want_f = a.get_populations()
        assert a.stats()["step"] == 2 * n
    with make_ctx(lb, lat, scheme, shape, storage=storage) as b:
        b.set_state(state)
        assert b.stats()["step"] == n
        b.step(n)
        got = b.get_state()
        got_f = b.get_populations()
        assert b.stats()["step"] == 2 * n
    assert got == want                       # header (step counter, hash) and raw buffer
    assert np.array_equal(got_f, want_f)


def test_restart_rejects_foreign_states():
    lb = library()
    shape = (64, 20, 12)
    m = oracle_model("D3Q19", "forcing")
    f0 = drop_populations(m, shape, 6.0)
    with make_ctx(lb, "D3Q19", "forcing", shape, storage=F16DEV) as a:
        a.set_populations(f0)
        a.step(3)
        state = a.get_state()
    bad = bytearray(state)
    bad[0] ^= 1
    others = [
        (dict(storage=F16DEV, T=0.54), state, "parameter hash"),
        (dict(storage=BF16DEV), state, "storage"),
        (dict(storage=F16DEV), state[:-2], "size"),
        (dict(storage=F16DEV), bytes(bad), "magic"),
    ]
    for kw, st, why in others:
        with make_ctx(lb, "D3Q19", "forcing", shape, **kw) as b:
            with pytest.raises(lb.LBError) as e:
                b.set_state(st)
            assert e.value.status == 1, why
    with make_ctx(lb, "D3Q19", "forcing", (64, 20, 10), storage=F16DEV) as b:
        with pytest.raises(lb.LBError):
            b.set_state(state)
    with make_ctx(lb, "D3Q19", "forcing", shape, storage=F16DEV) as b:
        with pytest.raises(lb.LBError) as e:
            b.get_state()                     # nothing to export before an init
        assert e.value.status == 6


@pytest.mark.parametrize("lat,scheme,shape,centre", [
    ("D2Q9", "equilibrium", (48, 40), (24.0, 20.0)),
    ("D2Q9", "forcing", (48, 40), (13.0, 30.0)),
    ("D3Q19", "forcing", (24, 20, 18), (12.0, 10.0, 9.0)),
])
def test_stats_dP_and_max_du_match_the_oracle(lat, scheme, shape, centre):
    """dP = p0(rho at the drop centre) - p0(rho at the farthest site) (Sec. IV)
    at the probes lb_init_drops chooses, and max|u(t) - u(t - 100)| between two
    lb_stats_get calls, both against the oracle's fields (float64, 1e-12)."""
    lb = library()
    m = oracle_model(lat, scheme)
    rl, rg = O.coexistence(m.a, m.b, m.T)
    nx, ny, nz = (tuple(shape) + (1,))[:3]
    R = 0.3 * min(shape)
    f = O.init_equilibrium(O.drop_density((nz, ny, nx), [centre], [R], rl, rg), m)
    with make_ctx(lb, lat, scheme, shape) as ctx:
        ctx.init_drops([centre], [R], 2.0)
        inside, outside = ctx.probes()
        c3 = (tuple(centre) + (0.0,))[:3]
        assert inside == tuple(int(round(v)) for v in c3)
        # farthest from the centre: the antipode (n/2 away on every axis)
        assert outside == tuple((int(round(c3[a])) + ([nx, ny, nz][a] // 2)) % [nx, ny, nz][a] if a < m.dim else 0
                                for a in range(3))
        ctx.step(200)
        s1 = ctx.stats()
        assert s1["max_du"] == -1.0 and s1["du_steps"] == 0
        ctx.step(100)
        s2 = ctx.stats()
    f1 = O.run(f, m, 200)
    f2 = O.run(f1, m, 100)
    _, _, u1 = O.moments(f1, m)
    _, _, u2 = O.moments(f2, m)
    du = float(np.sqrt(sum((a - b) ** 2 for a, b in zip(u2, u1))).max())
    cz, cy, cx = inside[2], inside[1], inside[0]
    fz, fy, fx = outside[2], outside[1], outside[0]
    d2 = O.diagnostics(f2, m, centre=(cz, cy, cx), far=(fz, fy, fx))
    assert s2["du_steps"] == 100
    assert du > 1e-9
    assert abs(s2["max_du"] - du) <= 1e-12 * max(du, 1e-3)
    assert abs(s2["dP"] - d2["dP"]) <= 1e-12
    assert d2["dP"] > 0                                    # higher pressure inside the drop


def test_set_probes_and_validation():
    lb = library()
    with make_ctx(lb, "D2Q9", "equilibrium", (16, 12)) as ctx:
        assert ctx.probes() == ((8, 6, 0), (0, 0, 0))
        ctx.set_probes((3, 4), (15, 11))
        assert ctx.probes() == ((3, 4, 0), (15, 11, 0))
        with pytest.raises(lb.LBError):
            ctx.set_probes((16, 4), (0, 0))
