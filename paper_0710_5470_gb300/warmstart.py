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
