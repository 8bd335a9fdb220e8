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
# sites a warm-started drop may move from the centre of its start before its
# run is handed back to the tanh start (the translation mode of the periodic
# lattice: a predicted start can set the drop moving, and a slowly moving drop
# passes the max|u(t) - u(t - every)| test)
DRIFT_LIMIT = 0.5


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


def _reflect(a: np.ndarray, ax: int) -> np.ndarray:
    """a[(n - x) mod n] along axis ax: the mirror image about the centre n/2."""
    return np.roll(np.flip(a, axis=ax), 1, axis=ax)


def symmetrize(rho: np.ndarray) -> np.ndarray:
    """The average of a density field over the symmetries of the lattice that
    fix the centre of the box (mirrors about n/2 on every axis and, for equal
    sides, the permutations of the axes), exactly symmetric: every site sums
    the values of its orbit in sorted order, so mirror sites get identical
    values.  A field that is symmetric only to rounding would drive the drop
    off the centre through the translation mode of the periodic lattice."""
    import itertools
    imgs = []
    axes = list(range(rho.ndim))
    perms = list(itertools.permutations(axes)) if len(set(rho.shape)) == 1 else [tuple(axes)]
    for perm in perms:
        b = np.transpose(rho, perm)
        for flips in itertools.product((False, True), repeat=rho.ndim):
            c = b
            for ax, f in enumerate(flips):
                if f:
                    c = _reflect(c, ax)
            imgs.append(c)
    st = np.sort(np.stack(imgs), axis=0)
    return st.sum(axis=0) / len(imgs)


def predict_start(ws, start, d, use_u=True, interface_only=True):
    """Network prediction (rho, u) for a drop from its tanh-start density,
    averaged over the lattice symmetries fixing the domain centre (so a
    symmetric start gives a symmetric prediction) and keeping the start's
    mass; u = 0 when use_u is False, and then the density is made exactly
    symmetric (symmetrize).  With interface_only the density correction is
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
        rho = symmetrize(rho)
    return rho, u


def steps_to_steady(instances, ws=None, storage=lb.F64, scheme=lb.FORCING, tol=1e-9, every=100,
                    max_steps=60000, stream=None, use_u=True, interface_only=True, self_test=None):
    """Steps to the convergence check per instance, from the tanh start
    (ws is None) or from the network's prediction (velocity set to zero when
    use_u is False); self_test = (rtol_u, tol_rho, hold) selects the
    self-contained test of lb_batch_set_self_test instead of tol."""
    with lb.Batch(instances, A_VDW, B_VDW, scheme=scheme, storage=storage, stream=stream) as bt:
        if self_test is not None:
            bt.set_self_test(*self_test)
        bt.init_drops(2.0)
        if ws is not None:
            for k, d in enumerate(instances):
                rho, u = predict_start(ws, bt.fields(k)[0], d, use_u, interface_only)
                bt.init_fields(k, rho, u)
        bt.autotune(5)
        steps, status, total = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
        final = [bt.fields(k) for k in range(len(instances))]
    steps, status = list(steps), list(status)
    if ws is not None:
        # runs whose drop left the centre of its start run again from the tanh
        # start; their steps add up
        # (and runs that failed: unstable or not converged, counted at max_steps)
        redo = [k for k, d in enumerate(instances) if status[k] != 0 or left_its_start(final[k][0], d)]
        if redo:
            s2, st2, f2 = steps_to_steady([instances[k] for k in redo], None, storage, scheme, tol, every,
                                          max_steps, stream, self_test=self_test)
            for j, k in enumerate(redo):
                spent = steps[k] if steps[k] >= 0 else max_steps
                steps[k] = spent + s2[j] if s2[j] >= 0 else s2[j]
                status[k], final[k] = st2[j], f2[j]
    return steps, status, final


def drop_centre(rho: np.ndarray) -> np.ndarray:
    """Centre of a drop on the periodic lattice, per axis (x, y[, z]): the
    argument of the first Fourier mode of rho - mean(rho) along the axis."""
    c = []
    for ax in range(rho.ndim - 1, -1, -1):
        n = rho.shape[ax]
        prof = (rho - rho.mean()).sum(axis=tuple(a for a in range(rho.ndim) if a != ax))
        ph = np.angle(np.sum(prof * np.exp(2j * np.pi * np.arange(n) / n)))
        c.append((ph % (2 * np.pi)) * n / (2 * np.pi))
    return np.array(c)


def settle(instances, finals, tol=1e-11, every=50, max_steps=200000, stream=None):
    """The steady states that the given converged states (rho, u) lead to:
    a float64 batch restarted from each (lb_batch_init_fields) and run until
    max|u(t) - u(t - every)| < tol.  Used to compare where two runs end up
    independently of where a looser stopping test left each of them."""
    with lb.Batch(instances, A_VDW, B_VDW, scheme=lb.FORCING, storage=lb.F64, stream=stream) as bt:
        bt.init_drops(2.0)
        for k, (rho, u) in enumerate(finals):
            bt.init_fields(k, rho, u)
        _, status, _ = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
        return [bt.fields(k) if status[k] == 0 else None for k in range(len(instances))]


def spans(rho: np.ndarray, rho_l: float, rho_g: float) -> list:
    """Per axis (x, y[, z]): whether the liquid (rho above the midpoint of the
    coexistence densities) reaches every coordinate along that axis - a stripe
    or slab across the periodic box rather than a drop.  A drop narrower than
    the box spans no axis."""
    liq = rho > 0.5 * (rho_l + rho_g)
    return [bool(liq.any(axis=tuple(a for a in range(rho.ndim) if a != ax)).all())
            for ax in range(rho.ndim - 1, -1, -1)]


def left_its_start(rho: np.ndarray, d) -> bool:
    """A run from a centred drop that must not be trusted: the drop moved more
    than DRIFT_LIMIT sites from the centre, or the liquid spans the box
    (the drop turned into a stripe or slab, another steady state of the
    periodic box)."""
    rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
    return drift_from_centre(rho) > DRIFT_LIMIT or any(spans(rho, rl, rg))


def drift_from_centre(rho: np.ndarray) -> float:
    """Distance (sites, periodic) of a drop's centre from the centre of the
    lattice (n/2 per axis), where every sweep drop starts."""
    n = np.array(rho.shape[::-1], dtype=float)
    d = (drop_centre(rho) - n / 2 + n / 2) % n - n / 2
    return float(np.sqrt((d ** 2).sum()))


def steady_observables(rho: np.ndarray, u: np.ndarray, rho_l: float, rho_g: float) -> dict:
    """Translation-invariant observables of a steady drop: the bulk densities
    (max and min of rho), the equimolar radius (from the excess mass over the
    vapour, a disc in 2D, a sphere in 3D) and the spurious velocity max|u|."""
    excess = float(((rho - rho_g) / (rho_l - rho_g)).sum())
    R = np.sqrt(excess / np.pi) if rho.ndim == 2 else (3.0 * excess / (4.0 * np.pi)) ** (1.0 / 3.0)
    return {"rho_max": float(rho.max()), "rho_min": float(rho.min()), "radius": float(R),
            "max_u": float(np.sqrt((u ** 2).sum(axis=0)).max())}


def same_steady_state(a, b, rho_l, rho_g, tol_rho=1e-4, tol_radius=1e-3, tol_u=0.02) -> dict:
    """Whether two steady drops (rho, u) are the same state of the same
    physics up to a translation of the periodic lattice: bulk densities within
    tol_rho, equimolar radii within tol_radius (relative) and max|u| within
    tol_u (relative).  Also returns the drop-centre displacement (sites) and
    the largest pointwise density difference, which a translation changes."""
    oa = steady_observables(a[0], a[1], rho_l, rho_g)
    ob = steady_observables(b[0], b[1], rho_l, rho_g)
    d = drop_centre(b[0]) - drop_centre(a[0])
    n = np.array(a[0].shape[::-1], dtype=float)
    d = (d + n / 2) % n - n / 2
    same = (abs(oa["rho_max"] - ob["rho_max"]) <= tol_rho and abs(oa["rho_min"] - ob["rho_min"]) <= tol_rho and
            abs(oa["radius"] - ob["radius"]) <= tol_radius * oa["radius"] and
            abs(oa["max_u"] - ob["max_u"]) <= tol_u * max(oa["max_u"], 1e-12))
    return {"same": bool(same), "shift": float(np.sqrt((d ** 2).sum())),
            "pointwise": float(np.abs(a[0] - b[0]).max()), "a": oa, "b": ob}


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


def predict_start3(ws3, start, d, use_u=False, interface_only=True):
    """Reflection-averaged network prediction (rho, u) of a D3Q19 drop from its
    tanh start; interface_only tapers the density correction as predict_start."""
    rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
    x = lb.ws_features(start, rl, rg, d["T"], d["kappa"], d["tau"], d["radius"])
    y = ws3.predict_sym(x)
    if interface_only:
        y[0] *= 1.0 - 4.0 * x[0] ** 2
    rho, u = lb.ws3_decode(start, rl, rg, y)
    if not use_u:
        u[:] = 0.0
        rho = symmetrize(rho)
    return rho, u


def steps_to_steady3(instances, ws3=None, storage=lb.F64, scheme=lb.FORCING, tol=1e-8, every=50, max_steps=40000,
                     settle_tol=None):
    """Steps to the convergence check per D3Q19 instance from the tanh start (ws3 None) or
    from the network's prediction; returns (steps, final (rho, u)), rho [z][y][x] and
    u [3][z][y][x] (None for an unstable run).  With settle_tol the run continues,
    uncounted, to that tighter tolerance before its final state is taken."""
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
                if settle_tol is not None and steps[-1] > 0:
                    run3_to_steady(ctx, settle_tol, every, 10 * max_steps)
                rho, u, _ = ctx.fields(want_v=False)
                final.append((rho.reshape(n, n, n), u.reshape(3, n, n, n)))
            except lb.LBError:
                steps.append(-2)
                final.append(None)
        if ws3 is not None and (steps[-1] <= 0 or left_its_start(final[-1][0], d)):
            # the run failed or the drop left the centre of its start: run again
            # from the tanh start, steps added (a failed run counts max_steps)
            s2, f2 = steps_to_steady3([d], None, storage, scheme, tol, every, max_steps, settle_tol)
            spent = steps[-1] if steps[-1] > 0 else max_steps
            steps[-1] = spent + s2[0] if s2[0] > 0 else s2[0]
            final[-1] = f2[0]
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
            rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
            c = same_steady_state(f_t[k], f_w[k], rl, rg)
            rows.append({"steps_tanh": s_t[k], "steps_warm": s_w[k], "same_steady": c["same"], "shift": c["shift"],
                         "pointwise": c["pointwise"],
                         "rms_err_tanh": float(np.sqrt(np.mean((start - f_t[k][0]) ** 2))),
                         "rms_err_warm": float(np.sqrt(np.mean((rho_w - f_t[k][0]) ** 2)))})
        out["held"].append({"side": side, "seconds_tanh": t_tanh, "seconds_warm": t_warm, "runs": rows})
    ws.close()
    return out


def evaluate_full(train_target=2000, held_count=128, train_side=64, held_side=256, epochs=200,
                  train_seed0=1, held_seed=999, storage=lb.F16DEV, self_test=(5e-4, 1e-5, 10), every=100,
                  max_steps=100000):
    """The warm start at full scale: a network trained on
    ``train_target`` solver-made steady states of drops drawn from the sweep
    ranges (T 0.50-0.56, kappa 0.002-0.03, tau 0.6-1.5, R 0.15-0.35 of the box;
    train_side^2 boxes; unstable draws skipped), evaluated on ``held_count``
    held-out drops of the same ranges on held_side^2 boxes.  Both starts run
    in one batch of the given storage to the self-contained steady test; per
    held-out drop: steps from either start, whether both reach the same steady
    state (same_steady_state: translation-invariant) and the drop's drift."""
    import time
    from . import inputs
    t0 = time.perf_counter()
    xs, ts, n_draw, seed = [], [], 0, train_seed0
    while sum(len(x) for x in xs) < train_target:
        inst = instances_from_sweep(inputs.sweep_instances(seed=seed, count=512, side=(train_side, train_side)))
        n_draw += len(inst)
        with lb.Batch(inst, A_VDW, B_VDW, scheme=lb.FORCING, storage=lb.F32) as bt:
            bt.set_self_test(*self_test)
            bt.init_drops(2.0)
            starts = [bt.fields(k)[0] for k in range(len(inst))]
            bt.autotune(5)
            _, status, _ = bt.run_to_steady(tol=1e-10, every=every, max_steps=max_steps)
            xb, tb = [], []
            for k, d in enumerate(inst):
                if status[k] != 0:
                    continue
                rho, u = bt.fields(k)
                rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
                xb.append(lb.ws_features(starts[k], rl, rg, d["T"], d["kappa"], d["tau"], d["radius"]))
                t = np.empty((3,) + rho.shape, dtype=np.float32)
                t[0] = (rho - starts[k]) / (rl - rg)
                t[1:] = 1e3 * u
                tb.append(t)
        xs.append(np.stack(xb))
        ts.append(np.stack(tb))
        seed += 1
    x = np.concatenate(xs)[:train_target]
    t = np.concatenate(ts)[:train_target]
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    ws, hist = train(x, t, epochs=epochs, batch=16, lr=1e-3)
    t_train = time.perf_counter() - t1
    held = instances_from_sweep(inputs.sweep_instances(seed=held_seed, count=held_count,
                                                       side=(held_side, held_side)))
    tp = time.perf_counter()
    s_t, st_t, f_t = steps_to_steady(held, None, storage=storage, every=every, max_steps=max_steps,
                                     self_test=self_test)
    sec_t = time.perf_counter() - tp
    tp = time.perf_counter()
    s_w, st_w, f_w = steps_to_steady(held, ws, storage=storage, every=every, max_steps=max_steps, use_u=False,
                                     self_test=self_test)
    sec_w = time.perf_counter() - tp
    ws.close()
    both_ok = [k for k in range(len(held)) if st_t[k] == 0 and st_w[k] == 0]
    t_settle = time.perf_counter()
    set_t = settle([held[k] for k in both_ok], [f_t[k] for k in both_ok])
    set_w = settle([held[k] for k in both_ok], [f_w[k] for k in both_ok])
    t_settle = time.perf_counter() - t_settle
    settled = {k: (set_t[j], set_w[j]) for j, k in enumerate(both_ok)}
    rows = []
    for k, d in enumerate(held):
        row = {"steps_tanh": int(s_t[k]), "steps_warm": int(s_w[k]), "status": [int(st_t[k]), int(st_w[k])]}
        if k in settled and settled[k][0] is not None and settled[k][1] is not None:
            rl, rg = lb.coexistence(A_VDW, B_VDW, d["T"])
            # where both runs end up: each final state settled in float64 to 1e-11
            c = same_steady_state(settled[k][0], settled[k][1], rl, rg)
            row.update(same=c["same"], shift=c["shift"], pointwise=c["pointwise"],
                       spans_tanh=spans(settled[k][0][0], rl, rg), spans_warm=spans(settled[k][1][0], rl, rg),
                       spans_stop=[spans(f_t[k][0], rl, rg), spans(f_w[k][0], rl, rg)],
                       d_rho_max=c["b"]["rho_max"] - c["a"]["rho_max"], d_rho_min=c["b"]["rho_min"] - c["a"]["rho_min"],
                       d_radius=c["b"]["radius"] - c["a"]["radius"],
                       max_u_rel=(c["b"]["max_u"] - c["a"]["max_u"]) / max(c["a"]["max_u"], 1e-300))
        rows.append(row)
    both = [r for r in rows if "same" in r]
    return {"train": {"samples": int(len(x)), "draws": n_draw, "side": train_side, "data_seconds": t_data,
                      "train_seconds": t_train, "epochs": epochs, "loss_first": float(hist[0]),
                      "loss_last": float(hist[-1])},
            "held": {"count": held_count, "side": held_side, "converged_both": len(both),
                     "same_steady": sum(r["same"] for r in both),
                     "steps_ratio": float(sum(r["steps_warm"] for r in both) / max(1, sum(r["steps_tanh"] for r in both))),
                     "seconds_tanh": sec_t, "seconds_warm_incl_inference": sec_w, "settle_seconds": t_settle,
                     "storage": storage, "self_test": list(self_test)},
            "runs": rows}


def steady_parameter_bound(sets=((48, 16, 11), (96, 16, 12)), tol=1e-9, every=100, max_steps=100000) -> dict:
    """What a start can gain that knows the steady bulk densities and radius
    exactly: for held-out drops (the warm start's ranges; side, count, seed
    per set), the steps to the float64 test from the tanh start of the
    coexistence densities and initial radius, against the steps from a tanh
    profile (width 2) with the run's own steady bulk densities (centre and
    corner site) and equimolar radius, scaled to the start's mass.  A ratio
    near 1 means the steps are spent settling the interface profile and the
    flow, not the radius or the bulk densities."""
    import math
    from . import inputs
    out = []
    for side, count, seed in sets:
        sw = inputs.sweep_instances(seed=seed, count=count, side=(side, side), T=(0.53, 0.56),
                                    kappa=(0.005, 0.015), tau=(0.7, 1.2), rfrac=(0.2, 0.35))
        inst = instances_from_sweep(sw)
        s_t, st_t, f_t = steps_to_steady(inst, None, tol=tol, every=every, max_steps=max_steps)
        y, x = np.mgrid[0:side, 0:side]
        dx = np.minimum(np.abs(x - side / 2), side - np.abs(x - side / 2))
        dy = np.minimum(np.abs(y - side / 2), side - np.abs(y - side / 2))
        dist = np.hypot(dx, dy)
        with lb.Batch(inst, A_VDW, B_VDW, scheme=lb.FORCING, storage=lb.F64) as bt:
            bt.init_drops(2.0)
            for k in range(count):
                rho = f_t[k][0].reshape(side, side)
                rl, rg = float(rho[side // 2, side // 2]), float(rho[0, 0])
                R = math.sqrt((float(rho.sum()) - rg * side * side) / (rl - rg) / math.pi)
                start = rg + (rl - rg) * 0.5 * (1 + np.tanh((R - dist) / 2.0))
                r0 = bt.fields(k)[0]
                start = start * (float(r0.sum()) / float(start.sum()))
                bt.init_fields(k, start.reshape(r0.shape), np.zeros((2,) + r0.shape))
            bt.autotune(5)
            s_p, st_p, _ = bt.run_to_steady(tol=tol, every=every, max_steps=max_steps)
        ok = [k for k in range(count) if st_t[k] == 0 and st_p[k] == 0]
        out.append({"side": side, "count": count, "converged_both": len(ok),
                    "steps_tanh": [int(s_t[k]) for k in ok], "steps_steady_parameters": [int(s_p[k]) for k in ok],
                    "ratio": float(np.sum([s_p[k] for k in ok]) / max(1, np.sum([s_t[k] for k in ok])))})
    return {"tol": tol, "every": every, "sets": out}


if __name__ == "__main__":
    import json
    import sys
    from . import build
    build.build()
    lb.load_library()
    if "full" in sys.argv:
        res = evaluate_full()
    elif "bound" in sys.argv:
        res = steady_parameter_bound()
    else:
        res = evaluate3()
    print(json.dumps(res), flush=True)
