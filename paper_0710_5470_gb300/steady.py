"""Time to steady state of a sweep of D2Q9 drop runs, driven through the C ABI.

Two ways to bring every instance of a sweep to its steady state:

* ``plain``: the float64 solver one instance at a time (a batch of one per
  run), tanh start;
* ``fast``: every instance in one batch (one launch per step for the whole
  sweep, CUDA-graph replay of ``every`` steps plus the check, autotuned tile),
  a reduced storage format, and optionally the learned warm start
  (lb_ws_* prediction of the steady density from the tanh start).

Steady-state tests (the paper defines none; Sec. IV runs to a fixed time):
``tol``: max|u(t) - u(t - every)| < tol, the float64 test; rounding of
reduced storage keeps this quantity above any useful tol, so the
equal-accuracy comparison uses the reference test of lb_batch_set_reference:
for ``hold`` (10) consecutive checks, max|u| within ``band`` (5%) of the
float64 steady max|u| and the bulk densities (max rho, min rho) within
``tol_rho`` of the float64 steady ones, applied to both ways alike.  The
test is blind to a translation of the drop: rounding noise of reduced
storage moves drops slowly on the periodic lattice (a neutral mode), which
changes no steady-state observable.

Both are timed on the wall clock from the creation of the solver state to
the last instance retired (set-up, inference and autotuning included).
``compare`` measures how close the fast steady states are to the float64
ones.  All arithmetic runs in the library; this module moves arrays between
the calls and reads the clock.

  python -m paper_0710_5470_gb300.steady [--count 16] [--warm]   (one JSON line)
  python -m paper_0710_5470_gb300.steady --sweep [--count 256]   (the whole sweep, batched ways only)
  python -m paper_0710_5470_gb300.steady --self-test [--sweep]   (no reference values: self-contained test)
  python -m paper_0710_5470_gb300.steady --throughput [--storage f16dev] [--steps 200]   (batched step rate)
  python -m paper_0710_5470_gb300.steady --single 2048 [--scheme forcing] [--storage f16dev]   (one lattice)
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lb
from . import warmstart as W


def _set_refs(bt, refs, band, tol_rho, hold):
    bt.set_band(band, tol_rho, hold)
    for k, (umax, rho_max, rho_min) in enumerate(refs):
        bt.set_reference(k, umax, rho_max, rho_min)


def plain(instances, tol=1e-10, every=100, max_steps=200000, scheme=lb.FORCING, refs=None, band=0.05,
          tol_rho=1e-3, hold=10, stream=None):
    """float64, one instance per batch, tanh start; the reference test with
    refs[k] = (umax, rho_max, rho_min) when refs is given, else the tol test.
    Returns wall time (s, total and per instance), per-instance steps,
    status, last-check max|u|, max rho, min rho and final (rho, u)."""
    steps, status, final, secs, umax, rmax, rmin = [], [], [], [], [], [], []
    t0 = time.perf_counter()
    for k, d in enumerate(instances):
        t1 = time.perf_counter()
        with lb.Batch([d], W.A_VDW, W.B_VDW, scheme=scheme, storage=lb.F64, stream=stream) as bt:
            if refs is not None:
                _set_refs(bt, [refs[k]], band, tol_rho, hold)
            bt.init_drops(2.0)
            s, st, _ = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
            steps.append(s[0])
            status.append(st[0])
            _, um, hi, lo = bt.last_check()
            umax.append(float(um[0]))
            rmax.append(float(hi[0]))
            rmin.append(float(lo[0]))
            final.append(bt.fields(0))
        secs.append(time.perf_counter() - t1)
    return {"seconds": time.perf_counter() - t0, "instance_seconds": secs, "steps": steps, "status": status,
            "umax": umax, "rho_max": rmax, "rho_min": rmin, "final": final}


# Self-contained steady-state test per storage format (lb_batch_set_self_test):
# (rtol of max|u|, tol of the bulk densities, consecutive checks), each per
# check of 100 steps.  Set above the late-time check-to-check changes measured
# on the first 16 sweep instances (forcing scheme, ~3e4 steps; GB300): max|u|
# float64 1.7e-5, float32 1.8e-4, fp16 deviations 1.4e-4, bf16 deviations
# ~1e-3; bulk densities 1e-6 (float32, fp16) to 1.5e-5 (bf16).
DRIFT_LIMIT = W.DRIFT_LIMIT

SELF_TEST = {"f64": (5e-4, 1e-5, 10), "f32": (5e-4, 1e-5, 10), "f16dev": (5e-4, 1e-5, 10),
             "bf16dev": (3e-3, 5e-5, 10)}


def fast(instances, storage=lb.F32, tol=1e-10, every=100, max_steps=200000, scheme=lb.FORCING, ws=None,
         refs=None, band=0.05, tol_rho=1e-3, hold=10, autotune_steps=5, stream=None, self_test=None):
    """All instances in one batch with the given storage, tanh start or the
    network's prediction (ws); reference test when refs is given.  Same
    return layout as ``plain`` plus the time of the warm-start prediction.
    With a warm start the tanh start stays the fallback: instances that went
    unstable or missed the test from the predicted start run again from the
    tanh start in a second batch; their steps and wall time add to the first
    (``fallback`` = how many)."""
    t0 = time.perf_counter()
    with lb.Batch(instances, W.A_VDW, W.B_VDW, scheme=scheme, storage=storage, stream=stream) as bt:
        if refs is not None:
            _set_refs(bt, refs, band, tol_rho, hold)
        if self_test is not None:
            bt.set_self_test(*self_test)
        bt.init_drops(2.0)
        t_pred = 0.0
        if ws is not None:
            tp = time.perf_counter()
            for k, d in enumerate(instances):
                rho, u = W.predict_start(ws, bt.fields(k)[0], d, use_u=False, interface_only=True)
                bt.init_fields(k, rho, u)
            t_pred = time.perf_counter() - tp
        if autotune_steps > 0:
            bt.autotune(autotune_steps)
        s, st, total = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
        seconds = time.perf_counter() - t0
        _, um, hi, lo = bt.last_check()
        final = [bt.fields(k) for k in range(len(instances))]
    s, st, um, hi, lo = list(s), list(st), list(um), list(hi), list(lo)
    failed = [k for k, v in enumerate(st) if v != 0] if ws is not None else []
    # a predicted start can set the drop moving (the translation mode of the
    # periodic lattice) or turn it into a stripe across the box (another steady
    # state): such runs (warmstart.left_its_start) are not trusted and run
    # again from the tanh start
    drifted = []
    if ws is not None:
        for k, d in enumerate(instances):
            if st[k] == 0 and W.left_its_start(final[k][0], d):
                drifted.append(k)
        failed = sorted(set(failed) | set(drifted))
    if failed:
        t1 = time.perf_counter()
        sub_refs = [refs[k] for k in failed] if refs is not None else None
        with lb.Batch([instances[k] for k in failed], W.A_VDW, W.B_VDW, scheme=scheme, storage=storage,
                      stream=stream) as bt:
            if sub_refs is not None:
                _set_refs(bt, sub_refs, band, tol_rho, hold)
            if self_test is not None:
                bt.set_self_test(*self_test)
            bt.init_drops(2.0)
            s2, st2, total2 = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
            seconds += time.perf_counter() - t1
            _, um2, hi2, lo2 = bt.last_check()
            for j, k in enumerate(failed):
                s[k] = (max_steps if s[k] < 0 else s[k]) + s2[j] if s2[j] >= 0 else s2[j]
                st[k], um[k], hi[k], lo[k] = st2[j], um2[j], hi2[j], lo2[j]
                final[k] = bt.fields(j)
        total += total2
    return {"seconds": seconds, "steps": s, "status": st, "umax": [float(v) for v in um],
            "rho_max": [float(v) for v in hi], "rho_min": [float(v) for v in lo], "final": final,
            "predict_seconds": t_pred, "batch_steps": total, "fallback": len(failed), "drifted": len(drifted)}


def _centre(rho):
    """Centre of the drop on the periodic lattice: argument of the first
    Fourier mode of rho - mean(rho) along each axis (x, y)."""
    c = []
    for ax, n in ((1, rho.shape[1]), (0, rho.shape[0])):
        prof = (rho - rho.mean()).sum(axis=1 - ax)
        ph = np.angle(np.sum(prof * np.exp(2j * np.pi * np.arange(n) / n)))
        c.append((ph % (2 * np.pi)) * n / (2 * np.pi))
    return np.array(c)


def compare(ref, run):
    """Per-instance accuracy of ``run`` against ``ref`` (results of plain or
    fast on the same instances), for the instances that converged in both
    (None otherwise): relative error of max|u|, errors of the bulk densities
    (max rho, min rho), the displacement of the drop centre (periodic
    distance, sites) and the largest pointwise density difference."""
    out = []
    for k, ((r0, u0), (r1, u1)) in enumerate(zip(ref["final"], run["final"])):
        if ref["status"][k] != 0 or run["status"][k] != 0:
            out.append(None)
            continue
        m0 = float(np.sqrt((u0 ** 2).sum(axis=0)).max())
        m1 = float(np.sqrt((u1 ** 2).sum(axis=0)).max())
        d = _centre(r1) - _centre(r0)
        n = np.array([r0.shape[1], r0.shape[0]])
        d = (d + n / 2) % n - n / 2
        out.append({"max_u_ref": m0, "max_u": m1, "max_u_rel_err": abs(m1 - m0) / m0,
                    "rho_max_err": abs(float(r1.max() - r0.max())), "rho_min_err": abs(float(r1.min() - r0.min())),
                    "shift": float(np.hypot(*d)), "rho_pointwise_err": float(np.abs(r1 - r0).max())})
    return out


def train_network(seeds=(1, 2, 3, 4), count=64, side=64, epochs=200, tol=1e-8, every=50, max_steps=40000):
    """A warm-start network trained on steady states of sweeps with the given
    seeds (sweep parameter ranges, lattices resized to side^2).  Returns the
    network, the training time (s) and the number of training samples."""
    from . import inputs
    t0 = time.perf_counter()
    inst = []
    for s in seeds:
        inst += W.instances_from_sweep(inputs.sweep_instances(seed=s, count=count), side=side)
    x, t, keep, _ = W.steady_dataset(inst, tol=tol, every=every, max_steps=max_steps)
    ws, _ = W.train(x, t, epochs=epochs, batch=16, lr=1e-3)
    return ws, time.perf_counter() - t0, len(keep)


def _summary(name, res, ref=None):
    ok = [k for k, s in enumerate(res["status"]) if s == 0]
    out = {"seconds": res["seconds"], "converged": len(ok), "instances": len(res["status"]),
           "mean_steps": float(np.mean([res["steps"][k] for k in ok])) if ok else None}
    if "predict_seconds" in res:
        out["predict_seconds"] = res["predict_seconds"]
    if ref is not None:
        c = [x for x in compare(ref, res) if x]
        if c:
            for key in ("max_u_rel_err", "rho_max_err", "rho_min_err", "shift", "rho_pointwise_err"):
                out[key + "_max"] = max(x[key] for x in c)
    return out


ARMS = {"f64": lb.F64, "f32": lb.F32, "f16dev": lb.F16DEV, "bf16dev": lb.BF16DEV}


def experiment(count=16, seed=0, every=100, max_steps=200000, band=0.05, tol_rho=1e-3, hold=10, warm=False,
               arms=("f64", "f32", "f16dev", "bf16dev")):
    """The time-to-steady comparison on the first ``count`` instances of a
    parameter sweep (inputs.sweep_instances(seed)): float64 runs to the tol
    test give the reference steady states; every way is then timed with the
    reference test on the instances whose float64 run converged."""
    from . import inputs
    inst_all = W.instances_from_sweep(inputs.sweep_instances(seed=seed, count=count))
    ref_all = plain(inst_all, tol=1e-10, every=every, max_steps=max_steps)
    ok = [k for k, s in enumerate(ref_all["status"]) if s == 0]
    inst = [inst_all[k] for k in ok]
    refs = [(ref_all["umax"][k], ref_all["rho_max"][k], ref_all["rho_min"][k]) for k in ok]
    ref = {key: [ref_all[key][k] for k in ok]
           for key in ("steps", "status", "umax", "rho_max", "rho_min", "final", "instance_seconds")}
    ref["seconds"] = float(sum(ref["instance_seconds"]))
    out = {"sweep": {"seed": seed, "count": count, "sites": int(sum(d["nx"] * d["ny"] for d in inst)),
                     "converged_f64": len(ok),
                     "unstable_f64": sum(s == 4 for s in ref_all["status"]),
                     "not_converged_f64": sum(s == 5 for s in ref_all["status"])},
           "test": {"tol_f64": 1e-10, "every": every, "band": band, "tol_rho": tol_rho, "hold": hold},
           "plain_f64_tol": _summary("plain_f64_tol", ref)}
    kw = dict(every=every, max_steps=max_steps, refs=refs, band=band, tol_rho=tol_rho, hold=hold)
    runs = {"plain_f64_ref": plain(inst, **kw)}
    for a in arms:
        runs["batch_" + a] = fast(inst, storage=ARMS[a], **kw)
    if warm:
        ws, t_train, n_train = train_network()
        runs["batch_f16dev_warm"] = fast(inst, storage=lb.F16DEV, ws=ws, **kw)
        out["training"] = {"seconds": t_train, "samples": n_train}
        ws.close()
    base = runs["plain_f64_ref"]["seconds"]
    for name, r in runs.items():
        out[name] = _summary(name, r, ref)
        out[name]["speedup_vs_plain_f64_ref"] = base / r["seconds"]
        out[name]["speedup_vs_plain_f64_tol"] = ref["seconds"] / r["seconds"]
    return out


def experiment_self(count=16, seed=0, every=100, max_steps=200000, arms=("f16dev", "f32", "bf16dev")):
    """Time to steady state with no reference values: plain float64 (one
    instance per batch, tanh start) to max|u(t) - u(t - every)| < 1e-10,
    against one batch per reduced format stopped by the format's own
    self-contained test (SELF_TEST, lb_batch_set_self_test).  Accuracy of the
    fast steady states afterwards against the float64 ones (compare), on the
    instances converged in both."""
    from . import inputs
    inst = W.instances_from_sweep(inputs.sweep_instances(seed=seed, count=count))
    ref = plain(inst, tol=1e-10, every=every, max_steps=max_steps)
    out = {"sweep": {"seed": seed, "count": count, "sites": int(sum(d["nx"] * d["ny"] for d in inst))},
           "test": {"tol_f64": 1e-10, "every": every, "self": {a: SELF_TEST[a] for a in arms}},
           "plain_f64_tol": _summary("plain_f64_tol", ref)}
    for a in arms:
        r = fast(inst, storage=ARMS[a], every=every, max_steps=max_steps, self_test=SELF_TEST[a])
        summ = _summary("batch_" + a, r, ref)
        summ["speedup_vs_plain_f64_tol"] = ref["seconds"] / r["seconds"]
        c = [x for x in compare(ref, r) if x]
        summ["within_5pct"] = sum(x["max_u_rel_err"] <= 0.05 for x in c)
        summ["compared"] = len(c)
        out["batch_" + a + "_self"] = summ
    return out


def _sweep_summary(res, sites):
    """Wall time, lattice updates done (sum over instances of the steps it ran
    x its sites; the whole batch for an instance stopped by the cap) and their
    rate, and the retirement counts of a batched run."""
    st = res["status"]
    # an instance still running at the cap reports -1 steps: it ran the whole batch
    ran = [int(n) if n >= 0 else int(res["batch_steps"]) for n in res["steps"]]
    lu = sum(n * int(k) for n, k in zip(ran, sites))
    ok = [k for k, s in enumerate(st) if s == 0]
    return {"seconds": res["seconds"], "instances": len(st), "converged": len(ok),
            "unstable": sum(s == 4 for s in st), "not_converged": sum(s == 5 for s in st),
            "lattice_updates": lu, "mlups": lu / res["seconds"] / 1e6, "batch_steps": res["batch_steps"],
            "mean_steps_converged": float(np.mean([res["steps"][k] for k in ok])) if ok else None}


def sweep(count=256, seed=0, every=100, max_steps=200000, band=0.05, tol_rho=1e-3, hold=10,
          arms=("f64", "f16dev", "f32")):
    """The whole parameter sweep (inputs.sweep_instances(seed, count)), one
    batch per way.  float64 to the tol test (max|du| < 1e-10 per ``every``
    steps, at most ``max_steps``) gives the reference steady states; each
    way in ``arms`` (float64 included, for the like-for-like comparison) then
    runs the instances that converged in float64 to the reference test.  Per way: wall time from solver creation to the last
    instance retired, lattice updates done and their rate, retirement counts,
    and (reduced storage) the accuracy against the float64 steady states."""
    from . import inputs
    inst = W.instances_from_sweep(inputs.sweep_instances(seed=seed, count=count))
    sites = [d["nx"] * d["ny"] for d in inst]
    f64 = fast(inst, storage=lb.F64, tol=1e-10, every=every, max_steps=max_steps)
    out = {"sweep": {"seed": seed, "count": count, "sites": int(sum(sites)), "every": every,
                     "max_steps": max_steps},
           "test": {"tol_f64": 1e-10, "band": band, "tol_rho": tol_rho, "hold": hold},
           "batch_f64_tol": _sweep_summary(f64, sites)}
    ok = [k for k, s in enumerate(f64["status"]) if s == 0]
    refs = [(f64["umax"][k], f64["rho_max"][k], f64["rho_min"][k]) for k in ok]
    ref = {"final": [f64["final"][k] for k in ok], "status": [0] * len(ok)}
    for a in arms:
        r = fast([inst[k] for k in ok], storage=ARMS[a], every=every, max_steps=max_steps, refs=refs, band=band,
                 tol_rho=tol_rho, hold=hold)
        summ = _sweep_summary(r, [sites[k] for k in ok])
        c = [x for x in compare(ref, r) if x]
        for key in ("max_u_rel_err", "rho_max_err", "rho_min_err"):
            summ[key + "_max"] = max(x[key] for x in c) if c else None
        out["batch_" + a + "_ref"] = summ
    return out


def sweep_self(count=256, seed=0, every=100, max_steps=200000, arms=("f16dev", "f32")):
    """The whole sweep without reference values: one float64 batch to
    max|u(t) - u(t - every)| < 1e-10 (the plain test), then one batch per
    reduced format stopped by its self-contained test (SELF_TEST); per way the
    wall time, lattice updates and retirement counts, and for the reduced
    formats the accuracy of their steady states against the float64 ones on
    the instances converged in both (max|u| within 5%: how many)."""
    from . import inputs
    inst = W.instances_from_sweep(inputs.sweep_instances(seed=seed, count=count))
    sites = [d["nx"] * d["ny"] for d in inst]
    f64 = fast(inst, storage=lb.F64, tol=1e-10, every=every, max_steps=max_steps)
    out = {"sweep": {"seed": seed, "count": count, "sites": int(sum(sites)), "every": every,
                     "max_steps": max_steps},
           "test": {"tol_f64": 1e-10, "self": {a: SELF_TEST[a] for a in arms}},
           "batch_f64_tol": _sweep_summary(f64, sites)}
    for a in arms:
        r = fast(inst, storage=ARMS[a], every=every, max_steps=max_steps, self_test=SELF_TEST[a])
        summ = _sweep_summary(r, sites)
        c = [x for x in compare(f64, r) if x]
        summ["compared"] = len(c)
        summ["within_5pct"] = sum(x["max_u_rel_err"] <= 0.05 for x in c)
        for key in ("max_u_rel_err", "rho_max_err", "rho_min_err"):
            summ[key + "_max"] = max(x[key] for x in c) if c else None
        summ["speedup_vs_f64_tol"] = f64["seconds"] / r["seconds"]
        out["batch_" + a + "_self"] = summ
    return out


def throughput(storage=lb.F16DEV, steps=200, count=256, seed=0, scheme=lb.FORCING, autotune_steps=5):
    """Batched step rate on the lattice sizes of the sweep
    (inputs.sweep_instances(seed, count)) at parameters where every instance
    is stable (T = 0.55, kappa = 0.01, tau = 1): wall clock around ``steps``
    steps after autotuning and 10 warm-up steps, closed by a read of the
    batch's check buffer (a stream synchronisation).  Returns the sites,
    the chosen tile and the rate in GLUPS."""
    from . import inputs
    inst = W.instances_from_sweep(inputs.sweep_instances(seed=seed, count=count))
    for d in inst:
        d.update(T=0.55, kappa=0.01, tau=1.0)
    sites = sum(d["nx"] * d["ny"] for d in inst)
    with lb.Batch(inst, W.A_VDW, W.B_VDW, scheme=scheme, storage=storage) as bt:
        bt.init_drops(2.0)
        tile = bt.autotune(autotune_steps) if autotune_steps > 0 else None
        bt.step(10)
        bt.last_check()
        t0 = time.perf_counter()
        bt.step(steps)
        bt.last_check()
        dt = time.perf_counter() - t0
    return {"instances": count, "sites": sites, "steps": steps, "tile": tile, "seconds": dt,
            "glups": sites * steps / dt / 1e9}


def single_throughput(n=2048, storage=lb.F16DEV, scheme=lb.FORCING, steps=400, warmup=100):
    """Step rate of one D2Q9 n x n lattice (a centred drop of radius n/4, T =
    0.55, kappa = 0.01, tau = 1): `steps` steps of one lb_step call after
    `warmup`, wall clock closed by a synchronisation; best of three.  Returns
    the kernel form and the rate in GLUPS."""
    with lb.Context(lb.D2Q9, (n, n), W.A_VDW, W.B_VDW, 0.55, 0.01, 1.0, scheme=scheme, storage=storage) as ctx:
        ctx.init_drops([(n / 2, n / 2)], [n / 4], 2.0)
        ctx.step(warmup)
        ctx.synchronize()
        best = None
        for _ in range(3):
            t0 = time.perf_counter()
            ctx.step(steps)
            ctx.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        form = ctx.kernel_info()["form"]
    return {"n": n, "scheme": "forcing" if scheme == lb.FORCING else "equilibrium", "steps": steps, "form": form,
            "seconds": best, "glups": n * n * steps / best / 1e9}


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--count", type=int, default=None, help="instances (default 16; 256 with --sweep)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--every", type=int, default=100)
    p.add_argument("--max-steps", type=int, default=200000)
    p.add_argument("--tol-rho", type=float, default=1e-3)
    p.add_argument("--warm", action="store_true")
    p.add_argument("--self-test", action="store_true",
                   help="no reference values: reduced formats stopped by their own test (experiment_self())")
    p.add_argument("--sweep", action="store_true",
                   help="the whole sweep (default 256 instances), one batch per way (sweep())")
    p.add_argument("--throughput", action="store_true",
                   help="batched step rate on the sweep's sizes at stable parameters (throughput())")
    p.add_argument("--single", type=int, default=0, metavar="N",
                   help="step rate of one D2Q9 N x N lattice (single_throughput())")
    p.add_argument("--scheme", default="forcing", choices=["forcing", "equilibrium"], help="scheme of --single")
    p.add_argument("--storage", default="f16dev", choices=list(ARMS), help="storage of --throughput / --single")
    p.add_argument("--steps", type=int, default=200, help="timed steps of --throughput / --single")
    a = p.parse_args()
    from . import build
    build.build()
    lb.load_library()
    if a.throughput:
        print(json.dumps(throughput(ARMS[a.storage], a.steps, a.count or 256, a.seed)), flush=True)
        return
    if a.single:
        sch = lb.FORCING if a.scheme == "forcing" else lb.EQUILIBRIUM
        print(json.dumps(single_throughput(a.single, ARMS[a.storage], sch, a.steps)), flush=True)
        return
    if a.sweep and a.self_test:
        print(json.dumps(sweep_self(a.count or 256, a.seed, a.every, a.max_steps)), flush=True)
        return
    if a.sweep:
        print(json.dumps(sweep(a.count or 256, a.seed, a.every, a.max_steps, tol_rho=a.tol_rho)), flush=True)
        return
    if a.self_test:
        print(json.dumps(experiment_self(a.count or 16, a.seed, a.every, a.max_steps)), flush=True)
        return
    print(json.dumps(experiment(a.count or 16, a.seed, a.every, a.max_steps, tol_rho=a.tol_rho, warm=a.warm)), flush=True)


if __name__ == "__main__":
    main()
