"""Spurious velocity scans of Secs. IV-V (Figs. 2 and 3), driven through the C ABI.

Fig. 2: each free parameter of the D2Q9 model (w^p_{5-8}, w^t_{5-8},
w^xx_{5-8}, B, D; lb_set_free_params) is varied alone, the others at the
optimum of Sec. III, and the spurious velocity max|u| of the equilibrium
scheme is recorded; Fig. 2(b): the coefficient F of the stencil of the body
force (Eq. 28) in the forcing scheme of Sec. VI, spurious velocity max|v|.
The paper scans quasi-statically; here each value is a run of its own from
the tanh start (same 10^4 steps).

The paper's drop (D2Q9 100^2, R = 25 at the centre, T = 0.56, kappa = 0.025,
tanh start of width 2) is run for 10^4 steps at each relaxation time, in
float64, with the equilibrium scheme (Sec. II-IV, spurious velocity max|u|)
and with the forcing scheme (Sec. VI, max|v|, v = u + g/(2 rho), Eq. 40).
Beside each point: the factor S(tau) = tau - 6 tau^2 + 6 tau^3 (Eq. 26) that
multiplies the O(d^3) stencil errors, zero at tau = 1/2 + 1/(2 sqrt 3).

Also the 512^2 multi-drop workload (1-8 drops, every (T, kappa) of the
sweep grid, both schemes, float32 and float64): throughput and spurious velocity.

Fig. 1: the steady flow around the paper's drop with the simple gradient
(B = 0) and with the optimum: eight vortices in the gas, and the reduction.

  python -m paper_0710_5470_gb300.scans tau|fig1|fig2|multidrop [--steps N] [--out DIR]   (one JSON line)
"""
from __future__ import annotations

import argparse
import json
import math

from . import lb

A_VDW, B_VDW = 9.0 / 49.0, 2.0 / 21.0
PAPER_DROP = dict(n=100, R=25.0, T=0.56, kappa=0.025, width=2.0)
TAUS = (0.55, 0.6, 0.65, 0.7, 0.75, 0.789, 0.85, 0.9, 1.0, 1.1, 1.25, 1.5, 1.75, 2.0)


def S(tau: float) -> float:
    """Eq. 26: (1/tau) sum_i i^3 z^(i-1), z = 1 - 1/tau."""
    return tau - 6 * tau ** 2 + 6 * tau ** 3


def spurious_velocity(scheme: int, tau: float, steps: int = 10000, drop=PAPER_DROP, storage=lb.F64) -> dict:
    """max|u| and max|v| of the drop after `steps` steps; spurious = None
    when the run went unstable (LB_EUNSTABLE)."""
    n = drop["n"]
    with lb.Context(lb.D2Q9, (n, n), A_VDW, B_VDW, drop["T"], drop["kappa"], tau, scheme=scheme,
                    storage=storage) as ctx:
        ctx.init_drops([(n / 2, n / 2)], [drop["R"]], drop["width"])
        ctx.step(steps)
        try:
            st = ctx.stats()
        except lb.LBError as e:
            return {"tau": tau, "max_u": None, "max_v": None, "status": e.status, "spurious": None}
    return {"tau": tau, "max_u": st["max_u"], "max_v": st["max_v"], "status": st["status"],
            "spurious": st["max_u"] if scheme == lb.EQUILIBRIUM else st["max_v"]}


OPTIMUM = dict(lb.OPTIMUM_FREE)
FIG2 = {
    "wp58": [0.0, 1 / 48, 1 / 24, 1 / 16, 1 / 12, 5 / 48, 1 / 8, 7 / 48, 1 / 6],
    "wt58": [0.0, 1 / 48, 1 / 24, 1 / 16, 1 / 12, 5 / 48, 1 / 8, 7 / 48, 1 / 6],
    "wxx58": [-1 / 12, -5 / 72, -1 / 18, -1 / 24, -1 / 36, -1 / 72, 0.0],
    "B": [0.0, 1 / 48, 1 / 24, 1 / 16, 1 / 12, 5 / 48, 1 / 8, 7 / 48],
    "D": [1 / 12, 1 / 8, 1 / 6, 5 / 24, 1 / 4],
}
# Fig. 2(b): the force-stencil coefficient F of the forcing scheme (Eq. 28; E = 1/2 - 2F)
FIG2_FORCING = {
    "F": [0.0, 1 / 48, 1 / 24, 1 / 16, 1 / 12, 5 / 48, 1 / 8, 7 / 48],
}


def free_param_point(param: str, value: float, scheme: int = lb.EQUILIBRIUM, steps: int = 10000, tau: float = 1.0,
                     drop=PAPER_DROP) -> dict:
    """Spurious velocity with one free parameter changed from the optimum."""
    n = drop["n"]
    with lb.Context(lb.D2Q9, (n, n), A_VDW, B_VDW, drop["T"], drop["kappa"], tau, scheme=scheme,
                    storage=lb.F64) as ctx:
        ctx.set_free_params(**{param: value})
        ctx.init_drops([(n / 2, n / 2)], [drop["R"]], drop["width"])
        ctx.step(steps)
        try:
            st = ctx.stats()
        except lb.LBError as e:
            return {"value": value, "spurious": None, "status": e.status}
    return {"value": value, "spurious": st["max_u"] if scheme == lb.EQUILIBRIUM else st["max_v"],
            "status": st["status"]}


def fig2_scans(scans=FIG2, steps: int = 10000, forcing_scans=FIG2_FORCING) -> dict:
    out = {"drop": dict(PAPER_DROP), "steps": steps, "optimum": OPTIMUM, "scans": {}}
    for scheme, group in ((lb.EQUILIBRIUM, scans), (lb.FORCING, forcing_scans)):
        for param, values in group.items():
            pts = [free_param_point(param, v, scheme=scheme, steps=steps) for v in values]
            ok = [p for p in pts if p["spurious"] is not None]
            best = min(ok, key=lambda p: p["spurious"]) if ok else None
            out["scans"][param] = {"scheme": "equilibrium" if scheme == lb.EQUILIBRIUM else "forcing",
                                   "points": pts, "argmin": best["value"] if best else None,
                                   "min_spurious": best["spurious"] if best else None,
                                   "predicted": OPTIMUM[param]}
    eq = [v["min_spurious"] for k, v in out["scans"].items() if v["scheme"] == "equilibrium" and v["min_spurious"]]
    fo = out["scans"].get("F", {}).get("min_spurious")
    if eq and fo:
        # Sec. VI: the forcing scheme at F = 1/12 against the best equilibrium-scheme point
        out["forcing_gain"] = min(eq) / fo
    return out


def flow_pattern(rho, u, rho_l: float, rho_g: float, nth: int = 720, modes: int = 12) -> dict:
    """Angular structure of the spurious flow around a centred 2D drop (Fig. 1):
    on a circle in the gas halfway between the equimolar radius R_e and the
    box edge, the radial velocity u_r(theta) and the vorticity dx u_y - dy u_x
    (central differences, periodic), sampled at nth angles by bilinear
    interpolation; their sign changes around the circle (a ring of N vortices
    gives N of each) and the amplitudes |sum u_r e^{-i m theta}| / nth of the
    angular modes m = 0 .. modes of the radial velocity."""
    import numpy as np
    rho = np.asarray(rho, dtype=np.float64).reshape(np.shape(rho)[-2:])
    ux = np.asarray(u[0], dtype=np.float64).reshape(rho.shape)
    uy = np.asarray(u[1], dtype=np.float64).reshape(rho.shape)
    ny, nx = rho.shape
    R_e = math.sqrt(float(np.sum(rho - rho_g)) / (rho_l - rho_g) / math.pi)
    r = R_e + 0.5 * (0.5 * min(nx, ny) - R_e)
    wz = 0.5 * (np.roll(uy, -1, axis=1) - np.roll(uy, 1, axis=1)) - 0.5 * (np.roll(ux, -1, axis=0) - np.roll(ux, 1, axis=0))

    def sample(f, x, y):
        x0, y0 = np.floor(x).astype(int), np.floor(y).astype(int)
        fx, fy = x - x0, y - y0
        g = lambda yy, xx: f[yy % ny, xx % nx]
        return ((1 - fx) * (1 - fy) * g(y0, x0) + fx * (1 - fy) * g(y0, x0 + 1) + (1 - fx) * fy * g(y0 + 1, x0)
                + fx * fy * g(y0 + 1, x0 + 1))

    th = 2 * math.pi * np.arange(nth) / nth
    # the drop is centred at (n/2, n/2) of the site grid
    xs, ys = nx / 2 + r * np.cos(th), ny / 2 + r * np.sin(th)
    ur = sample(ux, xs, ys) * np.cos(th) + sample(uy, xs, ys) * np.sin(th)
    om = sample(wz, xs, ys)
    def changes(a):
        sg = np.sign(a)
        for k in range(len(sg)):          # an exact zero keeps the sign before it
            if sg[k] == 0:
                sg[k] = sg[k - 1] if k > 0 else 1.0
        return int(np.sum(sg != np.roll(sg, 1)))
    amp = [float(abs(np.sum(ur * np.exp(-1j * m * th))) / nth) for m in range(modes + 1)]
    return {"R_e": R_e, "r_probe": r, "ur_sign_changes": changes(ur), "vorticity_sign_changes": changes(om),
            "ur_modes": amp, "dominant_mode": int(np.argmax(amp)), "max_u": float(np.sqrt(ux ** 2 + uy ** 2).max())}


def fig1(steps: int = 10000, standard: dict | None = None, drop=PAPER_DROP, out_dir: str | None = None) -> dict:
    """Fig. 1: the steady spurious flow of the paper's drop (equilibrium scheme,
    float64) with a standard choice - by default the simple central-difference
    gradient, B = 0 (Sec. IV) - and with the optimum of Sec. III: the flow
    pattern of each (flow_pattern) and the reduction of max|u|.  With out_dir,
    the fields go to fig1.npz and the speed |u| of each run to a greyscale
    PGM image (headless)."""
    import numpy as np
    standard = standard if standard is not None else {"B": 0.0}
    n = drop["n"]
    rl, rg = lb.coexistence(A_VDW, B_VDW, drop["T"])
    res, fields = {"drop": dict(drop), "steps": steps, "standard": standard}, {}
    for name, params in (("standard", standard), ("optimum", {})):
        with lb.Context(lb.D2Q9, (n, n), A_VDW, B_VDW, drop["T"], drop["kappa"], 1.0, scheme=lb.EQUILIBRIUM,
                        storage=lb.F64) as ctx:
            ctx.set_free_params(**params)
            ctx.init_drops([(n / 2, n / 2)], [drop["R"]], drop["width"])
            ctx.step(steps)
            rho, u, _ = ctx.fields(want_v=False)
        rho2, u2 = rho.reshape(n, n), u.reshape(2, n, n)
        fields[name] = (rho2, u2)
        res[name] = flow_pattern(rho2, u2, rl, rg)
    res["reduction"] = res["standard"]["max_u"] / res["optimum"]["max_u"]
    if out_dir:
        import os
        os.makedirs(out_dir, exist_ok=True)
        np.savez(os.path.join(out_dir, "fig1.npz"), **{f"{k}_rho": v[0] for k, v in fields.items()},
                 **{f"{k}_u": v[1] for k, v in fields.items()})
        for k, (_, u2) in fields.items():
            sp = np.sqrt((u2 ** 2).sum(axis=0))
            img = (255 * sp / max(sp.max(), 1e-300)).astype(np.uint8)[::-1]
            with open(os.path.join(out_dir, f"fig1_{k}_speed.pgm"), "wb") as fh:
                fh.write(f"P5 {n} {n} 255\n".encode())
                fh.write(img.tobytes())
    return res


def multi_drop_sweep(seed: int = 0, storages=(lb.F32, lb.F64), steps: int = 20000, n: int = 512, tau: float = 0.8,
                     Ts=(0.50, 0.53, 0.55), kappas=(0.004, 0.01, 0.02)) -> dict:
    """D2Q9 n^2 with 1-8 non-overlapping drops R ~ U[20, 80] (inputs.random_drops(seed)), every
    (T, kappa) pair, both schemes: throughput (wall clock around the steps, synchronised) and
    the spurious velocity (max|u| equilibrium, max|v| forcing) after `steps` steps."""
    import time
    from . import inputs
    centres, radii, _ = inputs.random_drops(seed, (n, n))
    out = {"n": n, "steps": steps, "tau": tau, "drops": len(radii), "runs": []}
    for storage in storages:
        for scheme in (lb.EQUILIBRIUM, lb.FORCING):
            for T in Ts:
                for kappa in kappas:
                    with lb.Context(lb.D2Q9, (n, n), A_VDW, B_VDW, T, kappa, tau, scheme=scheme,
                                    storage=storage) as ctx:
                        ctx.init_drops(centres, radii, 2.0)
                        spur, t0, dt = None, None, None
                        try:
                            ctx.step(10)
                            ctx.synchronize()
                            t0 = time.perf_counter()
                            ctx.step(steps)
                            ctx.synchronize()
                            dt = time.perf_counter() - t0
                            st = ctx.stats()
                            spur = st["max_u"] if scheme == lb.EQUILIBRIUM else st["max_v"]
                        except lb.LBError:       # unstable (LB_EUNSTABLE): the failed sync still ends the steps
                            if t0 is not None and dt is None:
                                dt = time.perf_counter() - t0
                    out["runs"].append({"storage": storage, "scheme": scheme, "T": T, "kappa": kappa,
                                        "mlups": n * n * steps / dt / 1e6 if dt else None, "spurious": spur})
    return out


def tau_sweep(taus=TAUS, steps: int = 10000) -> dict:
    out = {"drop": dict(PAPER_DROP), "steps": steps, "points": []}
    for t in taus:
        e = spurious_velocity(lb.EQUILIBRIUM, t, steps)
        f = spurious_velocity(lb.FORCING, t, steps)
        out["points"].append({"tau": t, "S": S(t), "equilibrium": e["spurious"], "forcing": f["spurious"],
                              "status": [e["status"], f["status"]]})
    out["S_zero"] = 0.5 + 0.5 / math.sqrt(3.0)
    return out


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("what", choices=["tau", "fig1", "fig2", "multidrop"])
    p.add_argument("--steps", type=int, default=10000)
    p.add_argument("--out", default=None, help="fig1: directory for fig1.npz and the PGM speed images")
    a = p.parse_args()
    from . import build
    build.build()
    lb.load_library()
    if a.what == "tau":
        res = tau_sweep(steps=a.steps)
    elif a.what == "fig1":
        res = fig1(steps=a.steps, out_dir=a.out)
    elif a.what == "fig2":
        res = fig2_scans(steps=a.steps)
    else:
        res = multi_drop_sweep(steps=a.steps)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
