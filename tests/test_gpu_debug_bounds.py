"""The index-checked build of the library (-DLB_DEBUG_BOUNDS, bounds.cuh).

Every global population access of the fused step kernels - the D3Q19 pair
kernels of both schemes in both population layouts, the D3Q19 tile kernel,
the D2Q9 pair and tile kernels of single lattices and of batches - runs with its site index tested
against the lattice.  On the tiny and ragged grids of the parity tests (tiles
cut by the lattice edge, lattices narrower than the halo, periodic wraps on
every face) no access may fall outside, and the checked kernels must give
bit for bit the results of the ordinary build.  The checked library runs in
a child process (LB_LIBRARY points the binding at it); nothing is made to
fail on purpose."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.helpers import drop_populations, library, make_ctx, oracle_model

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [
    ("D3Q19", "forcing", (68, 20, 12), 2), ("D3Q19", "forcing", (64, 16, 9), 2), ("D3Q19", "forcing", (2, 3, 3), 2),
    ("D3Q19", "forcing", (38, 13, 11), 3), ("D3Q19", "forcing", (96, 20, 7), 3), ("D3Q19", "forcing", (37, 13, 11), 2),
    ("D3Q19", "forcing", (38, 13, 11), 1), ("D3Q19", "equilibrium", (38, 13, 11), 2),
    ("D3Q19", "equilibrium", (64, 16, 9), 2), ("D3Q19", "equilibrium", (64, 10, 5), 1),
    ("D3Q19", "equilibrium", (2, 5, 3), 1), ("D3Q19", "forcing", (22, 20, 18), 0),
    ("D2Q9", "forcing", (45, 37), 1), ("D2Q9", "forcing", (46, 37), 2), ("D2Q9", "equilibrium", (2, 5), 3),
    ("D2Q9", "equilibrium", (66, 20), 0),
]
STEPS = 7


def run_cases():
    lb = library()
    out = {}
    for n, (lat, scheme, shape, storage) in enumerate(CASES):
        m = oracle_model(lat, scheme)
        f0 = drop_populations(m, shape, 0.3 * min(shape), perturb=1e-3, seed=6)
        with make_ctx(lb, lat, scheme, shape, storage=storage) as ctx:
            ctx.set_populations(f0)
            ctx.step(STEPS)
            out[f"case{n}"] = ctx.get_populations()
    inst = [dict(nx=64, ny=64, T=0.55, kappa=0.01, tau=1.0, radius=12.0),
            dict(nx=33, ny=47, T=0.54, kappa=0.012, tau=0.9, radius=9.0),
            dict(nx=2, ny=5, T=0.55, kappa=0.01, tau=1.0, radius=1.0)]
    for storage in (0, 2):
        with lb.Batch(inst, 9 / 49, 2 / 21, scheme=lb.FORCING, storage=storage) as bt:
            bt.init_drops(2.0)
            bt.step(STEPS)
            for k in range(len(inst)):
                out[f"batch{storage}_{k}"] = bt.populations(k)
    return out


CHILD = """
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
from tests import test_gpu_debug_bounds as T
from paper_0710_5470_gb300 import lb
out = T.run_cases()
np.savez({npz!r}, **out)
print(json.dumps(lb.debug_bounds()))
"""


def test_checked_kernels_stay_in_bounds_and_match(tmp_path):
    from paper_0710_5470_gb300 import build
    lib = build.build(debug=True)
    npz = str(tmp_path / "checked.npz")
    env = dict(os.environ, LB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, npz=npz)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    checked, violation = json.loads(r.stdout.strip().splitlines()[-1])
    assert checked is True
    assert violation == 0, hex(violation)
    lb = library()
    assert lb.debug_bounds() == (False, 0)          # the ordinary build has no checks
    got = np.load(npz)
    want = run_cases()
    for key, arr in want.items():
        assert np.array_equal(got[key], arr), key
