"""Learned warm start for D2Q9 drop runs, driven through the C ABI.

1. ``steady_dataset``: run a sweep of drops to their steady state with the
   batched solver (lb_batch_*) and pair each tanh-start density with its
   steady density and velocity.
2. ``train``: fit the network (lb_ws_*) on the GPU.
3. ``steps_to_steady``: count the steps the solver needs from the tanh start
   and from the network's prediction (lb_batch_init_fields), with the same
   convergence check.

All arithmetic runs in the library (solver kernels, network kernels, feature
and decoding routines); this module only moves arrays between the calls.
"""
from __future__ import annotations

import numpy as np

from . import lb

A_VDW, B_VDW = 9.0 / 49.0, 2.0 / 21.0


def instances_from_sweep(sweep, side=None):
    """lb_instance dicts from inputs.sweep_instances entries (optionally resized)."""
    out = []
    for d in sweep:
        n = side or d["n"]
        R = d["R"] * n / d["n"]
        out.append(dict(nx=n, ny=n, T=d["T"], kappa=d["kappa"], tau=d["tau"], radius=R))
    return out


def steady_dataset(instances, storage=lb.F64, scheme=lb.FORCING, tol=1e-9, every=100, max_steps=60000,
                   stream=None):
    """Steady states of the given instances.  Returns (x, t, keep, steps):
    network inputs and targets for the converged instances (float32
    [n][c][y][x]), their indices in ``instances`` and the steps each took."""
    with lb.Batch(instances, A_VDW, B_VDW, scheme=scheme, storage=storage, stream=stream) as bt:
        bt.init_drops(2.0)
        starts = [bt.fields(k)[0] for k in range(len(instances))]
        bt.autotune(5)
        steps, status, _ = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
        xs, ts, keep = [], [], []
        for k, d in enumerate(instances):
            if status[k] != 0:
                continue
            rho, u = bt.fields(k)
            rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
            x = lb.ws_features(starts[k], rl, rg, d["T"], d["kappa"], d["tau"], d["radius"])
            t = np.empty((3,) + rho.shape, dtype=np.float32)
            t[0] = (rho - starts[k]) / (rl - rg)
            t[1:] = 1e3 * u
            xs.append(x)
            ts.append(t)
            keep.append(k)
    if not xs:
        return None, None, [], steps
    return np.stack(xs), np.stack(ts), keep, steps


def train(x, t, epochs=60, batch=16, lr=2e-3, seed=0, stream=None):
    """A trained network (lb.WarmStart) and its per-epoch loss."""
    ws = lb.WarmStart(seed=seed, stream=stream)
    hist = ws.train(x, t, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return ws, hist


def predict_start(ws, start, d, use_u=True, interface_only=False):
    """Network prediction (rho, u) for a drop from its tanh-start density,
    averaged over the lattice symmetries fixing the domain centre (so a
    symmetric start gives a symmetric prediction) and keeping the start's
    mass; u = 0 when use_u is False.  With interface_only the density correction is
    tapered by 1 - 4 c^2 (c the normalised tanh density, +-1/2 in the bulk),
    so bulk densities stay at their coexistence values."""
    rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
    x = lb.ws_features(start, rl, rg, d["T"], d["kappa"], d["tau"], d["radius"])
    y = ws.predict_sym(x)
    if interface_only:
        y[0] *= 1.0 - 4.0 * x[0] ** 2
    rho, u = lb.ws_decode(start, rl, rg, y)
    if not use_u:
        u[:] = 0.0
    return rho, u


def steps_to_steady(instances, ws=None, storage=lb.F64, scheme=lb.FORCING, tol=1e-9, every=100,
                    max_steps=60000, stream=None, use_u=True, interface_only=False):
    """Steps to the convergence check per instance, from the tanh start
    (ws is None) or from the network's prediction (velocity set to zero when
    use_u is False)."""
    with lb.Batch(instances, A_VDW, B_VDW, scheme=scheme, storage=storage, stream=stream) as bt:
        bt.init_drops(2.0)
        if ws is not None:
            for k, d in enumerate(instances):
                rho, u = predict_start(ws, bt.fields(k)[0], d, use_u, interface_only)
                bt.init_fields(k, rho, u)
        bt.autotune(5)
        steps, status, total = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
        final = [bt.fields(k) for k in range(len(instances))]
    return steps, status, final


# ---------------------------------------------------------------- D3Q19 drops

def instances3_from_sweep(sweep, side):
    """(side^3 box, T, kappa, tau, R) dicts from inputs.sweep_instances entries, R scaled to the box."""
    return [dict(n=side, T=d["T"], kappa=d["kappa"], tau=d["tau"], radius=d["R"] * side / d["n"]) for d in sweep]


def run3_to_steady(ctx, tol=1e-8, every=50, max_steps=40000):
    """Steps until max|u(t) - u(t - every)| < tol (checked on the host every `every` steps);
    -1 if not reached within max_steps.  Raises LBError if the run goes unstable."""
    _, u_prev, _ = ctx.fields(want_v=False)
    steps = 0
    while steps < max_steps:
        ctx.step(every)
        steps += every
        _, u, _ = ctx.fields(want_v=False)
        if np.sqrt(((u - u_prev) ** 2).sum(axis=0)).max() < tol:
            return steps
        u_prev = u
    return -1


def _context3(d, storage, scheme):
    n = d["n"]
    return lb.Context(lb.D3Q19, (n, n, n), A_VDW, B_VDW, d["T"], d["kappa"], d["tau"], scheme=scheme,
                      storage=storage)


def steady_dataset3(instances, storage=lb.F64, scheme=lb.FORCING, tol=1e-8, every=50, max_steps=40000):
    """3D steady states: (x, t, keep, steps) as steady_dataset, volumes [n][c][z][y][x]."""
    xs, ts, keep, steps = [], [], [], []
    for k, d in enumerate(instances):
        n = d["n"]
        with _context3(d, storage, scheme) as ctx:
            ctx.init_drops([(n / 2,) * 3], [d["radius"]], 2.0)
            start = ctx.fields(want_v=False)[0].reshape(n, n, n)
            try:
                s = run3_to_steady(ctx, tol, every, max_steps)
            except lb.LBError:
                s = -2
            steps.append(s)
            if s < 0:
                continue
            rho, u, _ = ctx.fields(want_v=False)
        rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
        xs.append(lb.ws_features(start, rl, rg, d["T"], d["kappa"], d["tau"], d["radius"]))
        t = np.empty((4, n, n, n), dtype=np.float32)
        t[0] = (rho.reshape(n, n, n) - start) / (rl - rg)
        t[1:] = 1e3 * u.reshape(3, n, n, n)
        ts.append(t)
        keep.append(k)
    if not xs:
        return None, None, [], steps
    return np.stack(xs), np.stack(ts), keep, steps


def predict_start3(ws3, start, d, use_u=False):
    """Reflection-averaged network prediction (rho, u) of a D3Q19 drop from its tanh start."""
    rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
    y = ws3.predict_sym(lb.ws_features(start, rl, rg, d["T"], d["kappa"], d["tau"], d["radius"]))
    rho, u = lb.ws3_decode(start, rl, rg, y)
    if not use_u:
        u[:] = 0.0
    return rho, u


def steps_to_steady3(instances, ws3=None, storage=lb.F64, scheme=lb.FORCING, tol=1e-8, every=50, max_steps=40000):
    """Steps to the convergence check per D3Q19 instance from the tanh start (ws3 None) or
    from the network's prediction; returns (steps, final densities)."""
    steps, final = [], []
    for d in instances:
        n = d["n"]
        with _context3(d, storage, scheme) as ctx:
            ctx.init_drops([(n / 2,) * 3], [d["radius"]], 2.0)
            if ws3 is not None:
                start = ctx.fields(want_v=False)[0].reshape(n, n, n)
                rho, u = predict_start3(ws3, start, d)
                ctx.init_fields(rho, u)
            try:
                steps.append(run3_to_steady(ctx, tol, every, max_steps))
                final.append(ctx.fields(want_v=False)[0].reshape(n, n, n))
            except lb.LBError:
                steps.append(-2)
                final.append(None)
    return steps, final


SWEEP3 = dict(T=(0.53, 0.56), kappa=(0.005, 0.015), tau=(0.7, 1.2), rfrac=(0.2, 0.35))


def train3(x, t, epochs=600, batch=4, lr=3e-4, seed=0, stream=None):
    """A trained 3D network (lb.WarmStart3) and its per-epoch loss."""
    ws = lb.WarmStart3(seed=seed, stream=stream)
    hist = ws.train(x, t, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return ws, hist


def evaluate3(train_seed=21, train_count=64, train_side=32, held_seed=99, held=((48, 8), (96, 4)), tol=1e-8,
              every=50, max_steps=40000):
    """Train on solver-made steady states of train_side^3 drops, then compare the steps to
    the steady-state check from the tanh start and from the network's start on held-out drops
    of each (side, count), and the rms density error of both starts against the steady state."""
    import time
    from . import inputs
    t0 = time.perf_counter()
    train = instances3_from_sweep(inputs.sweep_instances(seed=train_seed, count=train_count,
                                                         side=(train_side, train_side), **SWEEP3), train_side)
    x, t, keep, _ = steady_dataset3(train, tol=tol, every=every, max_steps=max_steps)
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    ws, hist = train3(x, t)
    out = {"train": {"samples": len(keep), "side": train_side, "data_seconds": t_data,
                     "train_seconds": time.perf_counter() - t1, "loss_first": float(hist[0]),
                     "loss_last": float(hist[-1])}, "held": []}
    for side, count in held:
        inst = instances3_from_sweep(inputs.sweep_instances(seed=held_seed, count=count,
                                                            side=(train_side, train_side), **SWEEP3), side)
        tp = time.perf_counter()
        s_t, f_t = steps_to_steady3(inst, None, tol=tol, every=every, max_steps=max_steps)
        t_tanh = time.perf_counter() - tp
        tp = time.perf_counter()
        s_w, f_w = steps_to_steady3(inst, ws, tol=tol, every=every, max_steps=max_steps)
        t_warm = time.perf_counter() - tp
        rows = []
        for k, d in enumerate(inst):
            if f_t[k] is None or f_w[k] is None or s_t[k] < 0 or s_w[k] < 0:
                rows.append({"steps_tanh": s_t[k], "steps_warm": s_w[k]})
                continue
            n = d["n"]
            with _context3(d, lb.F64, lb.FORCING) as ctx:
                ctx.init_drops([(n / 2,) * 3], [d["radius"]], 2.0)
                start = ctx.fields(want_v=False)[0].reshape(n, n, n)
            rho_w, _ = predict_start3(ws, start, d)
            rows.append({"steps_tanh": s_t[k], "steps_warm": s_w[k],
                         "same_steady": bool(np.abs(f_t[k] - f_w[k]).max() < 1e-4),
                         "rms_err_tanh": float(np.sqrt(np.mean((start - f_t[k]) ** 2))),
                         "rms_err_warm": float(np.sqrt(np.mean((rho_w - f_t[k]) ** 2)))})
        out["held"].append({"side": side, "seconds_tanh": t_tanh, "seconds_warm": t_warm, "runs": rows})
    ws.close()
    return out


if __name__ == "__main__":
    import json
    from . import build
    build.build()
    lb.load_library()
    print(json.dumps(evaluate3()), flush=True)
