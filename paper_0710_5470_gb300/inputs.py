"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Random numbers only: a SplitMix64 stream (Steele, Lea & Flood 2014) mapped to
doubles in [0, 1), and the drop / parameter draws built from it.  No
arithmetic of the lattice Boltzmann method lives here, so the CUDA path and
the oracle can both consume these inputs.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15, then the published mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


def centred_drop(shape_xyz, radius: float):
    """One drop at the box centre (n/2 per axis): (centres, radii)."""
    return [tuple(n / 2.0 for n in shape_xyz)], [float(radius)]


def random_drops(seed: int, shape_xyz, n_min=1, n_max=8, r_min=20.0, r_max=80.0, width=2.0, max_rejects=10000):
    """1-8 non-overlapping drops with radii U[r_min, r_max] and uniform centres.

    A candidate is rejected when its periodic distance to an accepted drop is
    below R_j + R_k + 4*width; after ``max_rejects`` rejections the list stops
    short (the count is returned).
    """
    rng = SplitMix64(seed)
    want = rng.integer(n_min, n_max)
    centres, radii, rejects = [], [], 0
    while len(radii) < want and rejects < max_rejects:
        R = rng.uniform(r_min, r_max)
        c = tuple(rng.uniform(0.0, float(n)) for n in shape_xyz)
        ok = True
        for c2, R2 in zip(centres, radii):
            d2 = 0.0
            for a, n in enumerate(shape_xyz):
                dd = abs(c[a] - c2[a])
                dd = min(dd, n - dd)
                d2 += dd * dd
            if d2 < (R + R2 + 4 * width) ** 2:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(R)
        else:
            rejects += 1
    return centres, radii, rejects


def sweep_instances(seed: int = 0, count: int = 256, side=(64, 384), T=(0.50, 0.56), kappa=(0.002, 0.03),
                    tau=(0.6, 1.5), rfrac=(0.15, 0.35)):
    """Parameter sweep of independent D2Q9 drop runs (one centred drop each)."""
    rng = SplitMix64(seed)
    out = []
    for k in range(count):
        n = rng.integer(*side)
        out.append({"n": n, "T": rng.uniform(*T), "kappa": rng.uniform(*kappa), "tau": rng.uniform(*tau),
                    "R": rng.uniform(*rfrac) * n})
    return out


def noise(seed: int, shape) -> np.ndarray:
    """Uniform noise in [-1, 1) of the given shape (float64), numpy PCG64 seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=shape)
