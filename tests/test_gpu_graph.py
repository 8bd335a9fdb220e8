"""lb_step replays a captured CUDA graph of 64 steps for long runs: the
populations after lb_step(n) equal those after n calls of lb_step(1)
(ordinary launches) bit for bit, for both lattices, both schemes and the
storage formats, across repeated calls (graphs of both starting buffers)."""
import numpy as np
import pytest

from tests.helpers import library, make_ctx

pytestmark = pytest.mark.gpu

CASES = [
    ("D2Q9", "forcing", (96, 64), 2),
    ("D2Q9", "equilibrium", (64, 40), 0),
    ("D2Q9", "forcing", (33, 20), 1),
    ("D3Q19", "forcing", (40, 24, 16), 1),
    ("D3Q19", "forcing", (34, 16, 12), 2),
    ("D3Q19", "equilibrium", (32, 16, 8), 3),
]


@pytest.mark.parametrize("lat,scheme,shape,storage", CASES)
def test_graph_replay_matches_single_launches(lat, scheme, shape, storage):
    lb = library()
    dim = len(shape)
    R = 0.3 * min(shape)
    centre = [s / 2 for s in shape]
    runs = []
    for mode in ("graph", "single"):
        with make_ctx(lb, lat, scheme, shape, storage=storage, tau=0.8) as ctx:
            ctx.init_drops([centre], [R], 2.0)
            out = []
            for n in (150, 70, 200):
                if mode == "graph":
                    ctx.step(n)
                else:
                    for _ in range(n):
                        ctx.step(1)
                out.append(ctx.get_populations())
            runs.append(out)
    for a, b in zip(*runs):
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)
    assert dim in (2, 3)
