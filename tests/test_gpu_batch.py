"""Batched D2Q9 sweeps (lb_batch_*) through the C ABI.

An instance of a batch runs the same per-tile arithmetic as a single-lattice
context, so float64 results agree bit for bit whatever tile the autotuner
picks; one instance is also checked against the oracle.  Retirement by the
convergence check is compared with the same check done by hand.
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from tests.helpers import A_VDW, B_VDW, library, make_ctx, oracle_model, rel_inf

pytestmark = pytest.mark.gpu

INST = [dict(nx=40, ny=33, T=0.55, kappa=0.01, tau=0.8, radius=9.0),
        dict(nx=64, ny=64, T=0.53, kappa=0.012, tau=1.2, radius=15.0),
        dict(nx=19, ny=45, T=0.56, kappa=0.006, tau=0.65, radius=5.0)]


@pytest.mark.parametrize("scheme", ["equilibrium", "forcing"])
def test_batch_instances_match_single_contexts_bitwise(scheme):
    lb = library()
    sch = 0 if scheme == "equilibrium" else 1
    with lb.Batch(INST, A_VDW, B_VDW, scheme=sch, storage=lb.F64) as bt:
        bt.init_drops(2.0)
        f_init = [bt.populations(k) for k in range(len(INST))]
        bt.autotune(3)
        for k in range(len(INST)):
            assert np.array_equal(bt.populations(k), f_init[k])      # autotune restored the state
        bt.step(37)
        got = [bt.populations(k) for k in range(len(INST))]
    for k, d in enumerate(INST):
        with make_ctx(lb, "D2Q9", scheme, (d["nx"], d["ny"]), T=d["T"], kappa=d["kappa"], tau=d["tau"]) as ctx:
            ctx.init_drops([(d["nx"] / 2, d["ny"] / 2)], [d["radius"]])
            assert np.array_equal(ctx.get_populations(), f_init[k])
            ctx.step(37)
            assert np.array_equal(ctx.get_populations(), got[k])
    # oracle check on a parameter set where rounding perturbations do not grow
    # (at T = 0.52, kappa = 0.02, tau = 1.2 a 1e-16 perturbation reaches 1e-10
    # within 37 steps in the oracle itself: an unstable mode)
    d = INST[1]
    m = oracle_model("D2Q9", scheme, T=d["T"], kappa=d["kappa"], tau=d["tau"])
    want = O.run(f_init[1], m, 37)
    assert rel_inf(got[1], want) < 1e-12


def test_run_to_steady_retires_at_the_hand_check():
    """Retirement step = first multiple of `every` with max|u(t) - u(t-every)| < tol."""
    lb = library()
    inst = [dict(nx=32, ny=32, T=0.55, kappa=0.01, tau=1.0, radius=8.0),
            dict(nx=24, ny=40, T=0.54, kappa=0.015, tau=0.9, radius=6.0)]
    tol, every = 1e-7, 50
    with lb.Batch(inst, A_VDW, B_VDW, scheme=1, storage=lb.F64) as bt:
        bt.init_drops(2.0)
        steps, status, total = bt.run_to_steady(tol=tol, every=every, max_steps=20000)
    assert status == [0, 0]
    for k, d in enumerate(inst):
        with make_ctx(lb, "D2Q9", "forcing", (d["nx"], d["ny"]), T=d["T"], kappa=d["kappa"], tau=d["tau"]) as ctx:
            ctx.init_drops([(d["nx"] / 2, d["ny"] / 2)], [d["radius"]])
            uprev = np.zeros((2, d["ny"], d["nx"]))
            t = 0
            while True:
                ctx.step(every)
                t += every
                _, u, _ = ctx.fields(want_v=False)
                du = np.sqrt(((u - uprev) ** 2).sum(axis=0)).max()
                uprev = u
                if du < tol:
                    break
            assert steps[k] == t


def test_unstable_instance_is_retired_alone():
    """A NaN density in one instance marks it LB_EUNSTABLE; the others converge."""
    lb = library()
    inst = [dict(nx=24, ny=24, T=0.55, kappa=0.01, tau=1.0, radius=6.0),
            dict(nx=24, ny=24, T=0.55, kappa=0.01, tau=1.0, radius=6.0)]
    with lb.Batch(inst, A_VDW, B_VDW, scheme=0, storage=lb.F64) as bt:
        bt.init_drops(2.0)
        rho, _ = bt.fields(1)
        rho[3, 3] = np.nan
        bt.init_fields(1, rho)
        steps, status, total = bt.run_to_steady(tol=1e-6, every=20, max_steps=4000)
    assert status[0] == 0 and status[1] == 4


@pytest.mark.parametrize("scheme", ["forcing", "equilibrium"])
@pytest.mark.parametrize("storage", [1, 2, 3])
def test_reduced_storage_batch_matches_single_context(storage, scheme):
    """With 32-bit arithmetic a batch runs the pair kernel on every instance,
    aligned pairs for an even nx (40, 64) and site-by-site pairs for an odd nx
    (19), with the single-lattice contexts' 32 x 8 tile: bit for bit the
    single contexts' results."""
    lb = library()
    sch = 0 if scheme == "equilibrium" else 1
    with lb.Batch(INST, A_VDW, B_VDW, scheme=sch, storage=storage) as bt:
        bt.init_drops(2.0)
        bt.step(20)
        got = [bt.populations(k) for k in range(len(INST))]
    for k, d in enumerate(INST):
        with make_ctx(lb, "D2Q9", scheme, (d["nx"], d["ny"]), storage=storage, T=d["T"], kappa=d["kappa"],
                      tau=d["tau"]) as ctx:
            ctx.init_drops([(d["nx"] / 2, d["ny"] / 2)], [d["radius"]])
            ctx.step(20)
            assert ctx.kernel_info()["form"].startswith("pairs")
            assert np.array_equal(ctx.get_populations(), got[k]), k


def test_reference_test_stops_reduced_storage_at_float64_accuracy():
    """lb_batch_set_reference: float32 instances retire once, for 10 checks,
    max|u| is within 5% of the float64 steady max|u| and the bulk densities
    within 1e-3 of the float64 steady ones; the last-check values agree with
    the retired state's fields."""
    lb = library()
    inst = [dict(nx=32, ny=32, T=0.55, kappa=0.01, tau=1.0, radius=8.0),
            dict(nx=24, ny=40, T=0.54, kappa=0.015, tau=0.9, radius=6.0)]
    with lb.Batch(inst, A_VDW, B_VDW, scheme=1, storage=lb.F64) as bt:
        bt.init_drops(2.0)
        steps64, status64, _ = bt.run_to_steady(tol=1e-10, every=100, max_steps=100000)
        du, umax, hi, lo = bt.last_check()
        ref = [bt.fields(k) for k in range(len(inst))]
    assert status64 == [0, 0] and (du < 1e-10).all()
    for k in range(len(inst)):
        m = np.sqrt((ref[k][1] ** 2).sum(axis=0)).max()
        assert abs(umax[k] - m) <= 1e-12 * m
        assert hi[k] == ref[k][0].max() and lo[k] == ref[k][0].min()
    with lb.Batch(inst, A_VDW, B_VDW, scheme=1, storage=lb.F32) as bt:
        with pytest.raises(lb.LBError):
            bt.set_band(band=-1.0)
        with pytest.raises(lb.LBError):
            bt.set_reference(2, 1e-6)
        bt.set_band(band=0.05, tol_rho=1e-3, hold=10)
        for k in range(len(inst)):
            bt.set_reference(k, umax[k], hi[k], lo[k])
        bt.init_drops(2.0)
        steps32, status32, _ = bt.run_to_steady(tol=1e-10, every=100, max_steps=100000)
        _, um32, hi32, lo32 = bt.last_check()
        got = [bt.fields(k) for k in range(len(inst))]
    assert status32 == [0, 0]
    for k in range(len(inst)):
        assert abs(um32[k] - umax[k]) <= 0.05 * umax[k]
        assert abs(hi32[k] - hi[k]) <= 1e-3 and abs(lo32[k] - lo[k]) <= 1e-3
        assert 1000 <= steps32[k] <= 2 * steps64[k] + 1000
        assert abs(got[k][0].max() - hi32[k]) <= 1e-12 and abs(got[k][0].min() - lo32[k]) <= 1e-12


def test_maximum_instance_count_matches_single_contexts():
    """4096 instances (the API's maximum; work items hold the instance in 12
    bits): instances on both sides of 2048 step exactly like single contexts."""
    lb = library()
    base = dict(nx=16, ny=8, T=0.55, kappa=0.01, tau=1.0, radius=3.0)
    inst = [dict(base, T=0.54 + 0.02 * (k % 7) / 7, tau=0.8 + 0.05 * (k % 5)) for k in range(4096)]
    with lb.Batch(inst, A_VDW, B_VDW, scheme=1, storage=lb.F64) as bt:
        bt.init_drops(2.0)
        bt.step(12)
        got = {k: bt.populations(k) for k in (0, 2047, 2048, 4095)}
    for k, f in got.items():
        d = inst[k]
        with make_ctx(lb, "D2Q9", "forcing", (d["nx"], d["ny"]), T=d["T"], kappa=d["kappa"], tau=d["tau"]) as ctx:
            ctx.init_drops([(d["nx"] / 2, d["ny"] / 2)], [d["radius"]])
            ctx.step(12)
            assert np.array_equal(ctx.get_populations(), f), k


def test_whole_sweep_driver_small():
    """steady.sweep on the first 4 sweep instances: the float64 batch gives the
    references, the reduced-storage batches run the converged ones to the
    reference test; counts and update totals are consistent."""
    library()
    from paper_0710_5470_gb300 import steady
    res = steady.sweep(count=4, seed=0, max_steps=30000, arms=("f16dev",))
    f64, f16 = res["batch_f64_tol"], res["batch_f16dev_ref"]
    assert f64["instances"] == 4
    assert f64["converged"] + f64["unstable"] + f64["not_converged"] == 4
    assert f16["instances"] == f64["converged"]
    assert f64["lattice_updates"] > 0 and f64["mlups"] > 0
    if f16["converged"]:
        assert f16["max_u_rel_err_max"] < 0.1


class _NaNNetwork:
    """Stands in for a warm-start network whose prediction is unusable."""

    def predict_sym(self, x):
        return np.full((3,) + x.shape[1:], np.nan, dtype=np.float32)


def test_warm_start_falls_back_to_tanh_start():
    """An unusable predicted start makes its instances unstable; steady.fast
    reruns them from the tanh start and they reach the steady-state test."""
    library()
    from paper_0710_5470_gb300 import lb, steady
    inst = [dict(nx=48, ny=48, T=0.55, kappa=0.01, tau=1.0, radius=12.0),
            dict(nx=40, ny=56, T=0.54, kappa=0.012, tau=0.9, radius=10.0)]
    res = steady.fast(inst, storage=lb.F64, tol=1e-8, every=50, max_steps=40000, ws=_NaNNetwork(),
                      autotune_steps=0)
    assert res["fallback"] == 2
    assert res["status"] == [0, 0]
    ref = steady.fast(inst, storage=lb.F64, tol=1e-8, every=50, max_steps=40000, autotune_steps=0)
    assert ref["status"] == [0, 0] and ref["fallback"] == 0
    for k in range(2):
        assert res["steps"][k] >= ref["steps"][k]
        assert np.abs(res["final"][k][0] - ref["final"][k][0]).max() < 1e-6
