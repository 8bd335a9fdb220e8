"""Binary-fluid runs on the C ABI (lb_binary_*): drops of one phase in the other.

The model is the paper's liquid-gas construction carried over to an order
parameter phi (Sec. I names binary fluids; the equations are stated in
include/lb.h beside lb_binary_params).  Everything here is argument marshalling
and bookkeeping around library calls; every step runs in the CUDA kernels.

    python -m paper_0710_5470_gb300.binary run --n 1024 --storage f32 --steps 12
    python -m paper_0710_5470_gb300.binary laplace --n 96 --radius 20 --steps 20000
    python -m paper_0710_5470_gb300.binary throughput --n 2048 --steps 400
    python -m paper_0710_5470_gb300.binary throughput --dim 3 --n 128 --steps 200
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, lb

DEFAULT = {"A": -0.04, "B": 0.04, "kappa": 0.08, "Gamma": 1.0, "tau": 1.0, "tau_phi": 1.0}


def phi_star(A: float, B: float) -> float:
    """Bulk order parameter of the two phases, sqrt(-A/B)."""
    return float(np.sqrt(-A / B))


def interface_width(A: float, kappa: float) -> float:
    """Width w of the flat profile phi* tanh(x / w): sqrt(-2 kappa / A)."""
    return float(np.sqrt(-2.0 * kappa / A))


def surface_tension(A: float, B: float, kappa: float) -> float:
    """sigma = 4 kappa phi*^2 / (3 w) of the flat profile."""
    return 4.0 * kappa * phi_star(A, B) ** 2 / (3.0 * interface_width(A, kappa))


def drop_phi(n: int, radius: float, A: float, kappa: float, B: float = DEFAULT["B"], dim: int = 2) -> np.ndarray:
    """phi of a centred drop of phase +phi* in -phi* on an n^dim periodic lattice
    (tanh profile of width w, periodic minimum-image distance)."""
    ax = np.arange(n, dtype=np.float64)
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    d2 = np.zeros((n,) * dim)
    for g in grids:
        dd = np.abs(g - n / 2)
        d2 += np.minimum(dd, n - dd) ** 2
    return phi_star(A, B) * np.tanh((radius - np.sqrt(d2)) / interface_width(A, kappa))


def context(n: int, scheme: str = "forcing", storage: str = "f32", params: dict | None = None, stream=None,
            dim: int = 2):
    p = dict(DEFAULT, **(params or {}))
    return lb.BinaryContext((n,) * dim, p["A"], p["B"], p["kappa"], p["Gamma"], p["tau"], p["tau_phi"],
                            scheme=lb.FORCING if scheme == "forcing" else lb.EQUILIBRIUM,
                            storage=lb.STORAGE_NAMES[storage], stream=stream)


def run(n: int, steps: int, scheme: str = "forcing", storage: str = "f32", radius: float | None = None,
        params: dict | None = None, dim: int = 2) -> dict:
    """A drop of radius n/4 (default) at rho = 1, `steps` steps; the context's statistics."""
    p = dict(DEFAULT, **(params or {}))
    with context(n, scheme, storage, p, dim=dim) as c:
        c.init_fields(np.ones((n,) * dim),
                      drop_phi(n, radius if radius else n / 4, p["A"], p["kappa"], p["B"], dim))
        c.step(steps)
        return c.stats()


def laplace(n: int, radius: float, steps: int, scheme: str = "forcing", storage: str = "f64",
            params: dict | None = None, dim: int = 2) -> dict:
    """Laplace's law: dP R_e / ((dim - 1) sigma) after `steps` steps (R_e the
    equimolar radius of phi, dP the bulk-pressure jump p0(centre) - p0(corner)),
    with max|v|."""
    p = dict(DEFAULT, **(params or {}))
    with context(n, scheme, storage, p, dim=dim) as c:
        c.init_fields(np.ones((n,) * dim), drop_phi(n, radius, p["A"], p["kappa"], p["B"], dim))
        c.step(steps)
        rho, phi, u, v, mu = c.fields()
    p0 = lambda r, f: r / 3.0 + 0.5 * p["A"] * f ** 2 + 0.75 * p["B"] * f ** 4
    c0 = (n // 2,) * dim
    corner = (0,) * dim
    pin, pout = phi[c0], phi[corner]
    excess = (phi.sum() - pout * n ** dim) / (pin - pout)
    r_e = float(np.sqrt(excess / np.pi) if dim == 2 else (3 * excess / (4 * np.pi)) ** (1 / 3))
    dP = float(p0(rho[c0], pin) - p0(rho[corner], pout))
    return {"n": n, "dim": dim, "radius": radius, "steps": steps, "scheme": scheme, "storage": storage, "R_e": r_e,
            "dP": dP, "dP_R_over_sigma": dP * r_e / ((dim - 1) * surface_tension(p["A"], p["B"], p["kappa"])),
            "max_v": float(np.sqrt((v ** 2).sum(axis=0)).max()), "mu_spread": float(mu.max() - mu.min())}


def throughput(n: int, steps: int, scheme: str = "forcing", storage: str = "f32", warmup: int = 64,
               dim: int = 2) -> dict:
    """Step rate (GLUPS) of the step, timed with CUDA events on the context's
    stream (graph replay of 64-step blocks)."""
    import torch
    stream = torch.cuda.Stream()
    p = DEFAULT
    with context(n, scheme, storage, stream=stream.cuda_stream, dim=dim) as c:
        c.init_fields(np.ones((n,) * dim), drop_phi(n, n / 4, p["A"], p["kappa"], p["B"], dim))
        c.step(warmup)
        c.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = c.stats()
    q = 9 if dim == 2 else 19
    # f and g read and written: every population in float32 / float64; with fp16
    # deviations f_0 and g_0 in float32 and the other 2 Q - 2 in fp16
    bpl = {"f32": 2 * 2 * q * 4, "f64": 2 * 2 * q * 8, "f16dev": 2 * (2 * 4 + (2 * q - 2) * 2)}[storage]
    sites = n ** dim
    return {"n": n, "dim": dim, "scheme": scheme, "storage": storage, "steps": steps, "ms_per_step": ms / steps,
            "glups": sites * steps / (ms / 1e3) / 1e9, "gbs": bpl * sites * steps / (ms / 1e3) / 1e9,
            "bytes_per_lu": bpl,
            "max_v": st["max_v"], "status": st["status"]}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("what", choices=["run", "laplace", "throughput"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--radius", type=float, default=None)
    ap.add_argument("--scheme", choices=["forcing", "equilibrium"], default="forcing")
    ap.add_argument("--storage", choices=["f64", "f32", "f16dev"], default="f32")
    ap.add_argument("--dim", type=int, choices=[2, 3], default=2, help="2: D2Q9, 3: D3Q19")
    a = ap.parse_args(argv)
    build.build()
    lb.load_library()
    t0 = time.perf_counter()
    if a.what == "run":
        out = run(a.n, a.steps, a.scheme, a.storage, a.radius, dim=a.dim)
    elif a.what == "laplace":
        out = laplace(a.n, a.radius or a.n / 4, a.steps, a.scheme, a.storage, dim=a.dim)
    else:
        out = throughput(a.n, a.steps, a.scheme, a.storage, dim=a.dim)
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out))


if __name__ == "__main__":
    main()
