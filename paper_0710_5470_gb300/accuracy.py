"""Accuracy of the reduced storage formats on the D3Q19 drop, driven through the C ABI.

Runs the same drop (tanh start, forcing scheme) for the same number of
steps in float64 and in each reduced format, and compares the spurious
velocity max|v| (v = u + g/(2 rho), Eq. 40), the velocity field and the
density field with the float64 run.  The float64 path is the one checked
against the oracle to 1e-12 per step on small lattices; at 128^3 it stands
in for the oracle, which would need hours per 1000 steps.

  python -m paper_0710_5470_gb300.accuracy [--edge 128] [--steps 10000]   (one JSON line)
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lb

A_VDW, B_VDW = 9.0 / 49.0, 2.0 / 21.0


def run(storage, edge=128, steps=10000, T=0.55, kappa=0.01, tau=1.0, radius=None, width=2.0):
    """(rho, v, seconds) after `steps` steps of the centred drop in the given storage."""
    R = 30.0 * edge / 128 if radius is None else radius
    with lb.Context(lb.D3Q19, (edge,) * 3, A_VDW, B_VDW, T, kappa, tau, scheme=lb.FORCING,
                    storage=lb.STORAGE_NAMES[storage]) as ctx:
        ctx.init_drops([(edge / 2,) * 3], [R], width)
        t0 = time.perf_counter()
        ctx.step(steps)
        ctx.synchronize()
        dt = time.perf_counter() - t0
        rho, _, v = ctx.fields()
    return rho, v, dt


def drift(rho_ref: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """Translation (sites, per axis z, y, x) that maps rho_ref onto rho, from
    the phase of the first Fourier mode of each axis: a field moved by d on a
    periodic axis of n sites has its first mode turned by -2 pi d / n."""
    d = np.zeros(rho.ndim)
    for ax in range(rho.ndim):
        n = rho.shape[ax]
        k = np.exp(-2j * np.pi * np.arange(n) / n)
        shape = [1] * rho.ndim
        shape[ax] = n
        k = k.reshape(shape)
        a0 = np.sum((rho_ref - rho_ref.mean()) * k)
        a1 = np.sum((rho - rho.mean()) * k)
        d[ax] = -np.angle(a1 / a0) * n / (2 * np.pi) if abs(a0) > 0 else 0.0
    return d


def shift(rho: np.ndarray, d) -> np.ndarray:
    """rho translated by -d (periodic, spectral interpolation)."""
    F = np.fft.fftn(rho)
    for ax, dd in enumerate(d):
        n = rho.shape[ax]
        k = np.fft.fftfreq(n) * n
        shape = [1] * rho.ndim
        shape[ax] = n
        F = F * np.exp(2j * np.pi * k * dd / n).reshape(shape)
    return np.real(np.fft.ifftn(F))


def compare(rho0, v0, rho, v, rho_l, rho_g) -> dict:
    """Errors of a reduced-storage run (rho, v) against the float64 run
    (rho0, v0): spurious velocity, pointwise density (relative per site),
    bulk densities (extremes), the drop's translation and the density error
    left after undoing it, and the error in the bulk phases (sites further
    than 45% of the density contrast from the interface midpoint)."""
    vmag0 = np.sqrt((v0 ** 2).sum(axis=0))
    vmag = np.sqrt((v ** 2).sum(axis=0))
    d = drift(rho0, rho)
    aligned = shift(rho, d)
    mid, half = 0.5 * (rho_l + rho_g), 0.5 * (rho_l - rho_g)
    bulk = np.abs(rho0 - mid) > 0.9 * half
    rel = np.abs(rho - rho0) / rho0
    return {"max_v": float(vmag.max()),
            "max_v_rel_err": float(abs(vmag.max() - vmag0.max()) / vmag0.max()),
            "v_field_err_rel": float(np.abs(v - v0).max() / vmag0.max()),
            "rho_pointwise_rel_err": float(rel.max()),
            "rho_bulk_sites_rel_err": float(rel[bulk].max()),
            "rho_extremes_rel_err": max(abs(float(rho.max() - rho0.max())) / float(rho0.max()),
                                        abs(float(rho.min() - rho0.min())) / float(rho0.min())),
            "drift_sites": [float(x) for x in d],
            "rho_aligned_rel_err": float((np.abs(aligned - rho0) / rho0).max())}


def storage_accuracy(edge=128, steps=10000, storages=("f32", "f16dev", "bf16dev")):
    rho0, v0, dt0 = run("f64", edge, steps)
    rl, rg = lb.coexistence(A_VDW, B_VDW, 0.55)
    vmag0 = np.sqrt((v0 ** 2).sum(axis=0))
    out = {"workload": f"D3Q19 {edge}^3, one centred drop R={30.0 * edge / 128:g}, forcing, T=0.55, kappa=0.01, "
                       f"tau=1.0, {steps} steps from the tanh start",
           "f64": {"max_v": float(vmag0.max()), "seconds": dt0}}
    for s in storages:
        rho, v, dt = run(s, edge, steps)
        out[s] = dict(compare(rho0, v0, rho, v, rl, rg), seconds=dt)
    return out


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--edge", type=int, default=128)
    p.add_argument("--steps", type=int, default=10000)
    a = p.parse_args()
    from . import build
    build.build()
    lb.load_library()
    print(json.dumps(storage_accuracy(a.edge, a.steps)), flush=True)


if __name__ == "__main__":
    main()
