"""Parity at the largest lattices: site indices near the 32-bit limit, byte offsets far past 4 GB.

The kernels index sites with 32-bit integers (lb_create refuses more than
2^31 - 1 sites) and address bytes with 64-bit offsets.  Two fp16-deviation
lattices, forcing scheme: D3Q19 1024^3 (1.07 G sites, 86 GB of populations)
and D2Q9 46000^2 (2.12 G sites, 98.5% of the 32-bit range, 85 GB).  Their
populations are too large to read back whole, so the check reads periodic
boxes (lb_get_populations_box) before and after one step: the oracle steps
each box on its own (periodic in the box, so wrong within 3 sites of the box
faces: the step at r reads populations within 3 sites) and the interior is
compared with the GPU's step, to the one-step bound of the 16-bit format
(1e-4 of the largest population).  Boxes sit on the drop's interface, across
the periodic corner (the largest indices next to the smallest) and at the
last sites of the lattice.
"""
import numpy as np
import pytest

from oracle import lb_oracle as O
from tests.helpers import A_VDW, B_VDW, library, rel_inf

pytestmark = pytest.mark.gpu

T, KAPPA, TAU, B, M = 0.55, 0.01, 1.0, 14, 3


def test_population_box_matches_whole_readback():
    lb = library()
    for shape in ((40, 24, 16), (34, 18)):
        lat = lb.D3Q19 if len(shape) == 3 else lb.D2Q9
        with lb.Context(lat, shape, A_VDW, B_VDW, T, KAPPA, TAU, scheme=lb.FORCING, storage=2) as ctx:
            ctx.init_drops([[s / 2 for s in shape]], [0.3 * min(shape)], 2.0)
            ctx.step(3)
            f = ctx.get_populations()
            for origin, size in (((0,) * len(shape), (5,) * len(shape)), (tuple(s - 3 for s in shape), (7,) * len(shape)),
                                 (tuple(s // 2 for s in shape), shape)):
                box = ctx.get_populations_box(origin, size)
                o = (tuple(origin) + (0,))[:3]
                b = (tuple(size) + (1,))[:3]
                iz = (o[2] + np.arange(b[2])) % f.shape[1]
                iy = (o[1] + np.arange(b[1])) % f.shape[2]
                ix = (o[0] + np.arange(b[0])) % f.shape[3]
                want = f[:, iz][:, :, iy][:, :, :, ix]
                assert np.array_equal(box, want)
            with pytest.raises(lb.LBError):
                ctx.get_populations_box((0,) * len(shape), tuple(s + 1 for s in shape))
            with pytest.raises(lb.LBError):
                ctx.get_populations_box((-1,) + (0,) * (len(shape) - 1), (2,) * len(shape))


def _need_device_bytes(nbytes):
    """Skip (not fail) when the GPU has less free memory than the lattice needs."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 1.05 * nbytes:
        pytest.skip(f"needs {nbytes / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")


def _check_boxes(lb, lat, shape, origins):
    dim = len(shape)
    sites = int(np.prod(shape))
    # fp16 deviations: 2 buffers of (4 + 2 (Q - 1)) bytes per site, plus the float64 density
    q = 19 if dim == 3 else 9
    _need_device_bytes(sites * (2 * (4 + 2 * (q - 1)) + 8))
    m = O.Model("D3Q19" if dim == 3 else "D2Q9", A_VDW, B_VDW, T, KAPPA, TAU, scheme="forcing")
    with lb.Context(lat, shape, A_VDW, B_VDW, T, KAPPA, TAU, scheme=lb.FORCING, storage=2) as ctx:
        ctx.init_drops([[s / 2 for s in shape]], [0.3 * min(shape)], 2.0)
        ctx.step(2)
        before = [ctx.get_populations_box(o, (B,) * dim) for o in origins]
        ctx.step(1)
        after = [ctx.get_populations_box(o, (B,) * dim) for o in origins]
    inner = (slice(None),) + ((slice(M, B - M),) * 3 if dim == 3 else (slice(None), slice(M, B - M), slice(M, B - M)))
    for o, f0, f1 in zip(origins, before, after):
        want = O.step(f0, m)
        err = rel_inf(f1[inner], want[inner])
        assert np.isfinite(f1).all()
        assert err < 1e-4, (o, err)


def test_d3q19_1024_cubed():
    lb = library()
    n = 1024
    R = 0.3 * n
    origins = [(int(n / 2 + R) - B // 2, n // 2 - B // 2, n // 2 - B // 2),    # interface, +x
               (n // 2 - B // 2, n // 2 - B // 2, int(n / 2 - R) - B // 2),    # interface, -z
               (n - B // 2, n - B // 2, n - B // 2),                            # across the periodic corner
               (n - B, n - B, n - B)]                                           # the last sites
    _check_boxes(lb, lb.D3Q19, (n, n, n), origins)


def test_d2q9_46000_squared():
    lb = library()
    n = 46000
    R = 0.3 * n
    origins = [(int(n / 2 + R) - B // 2, n // 2 - B // 2),
               (n // 2 - B // 2, int(n / 2 - R) - B // 2),
               (n - B // 2, n - B // 2),
               (n - B, n - B)]
    _check_boxes(lb, lb.D2Q9, (n, n), origins)


@pytest.mark.parametrize("n,cuts", [(256, (64, 128, 192)), (224, (74, 149))], ids=["256c4", "224c3"])
def test_d3q19_uniform_chunks_across_chunk_boundaries(n, cuts):
    """Lattices with fewer than two resident slots per tile (224^3, 256^3 on 152 SMs) split
    every column into equal z chunks; boxes straddling the chunk boundaries (and the drop
    interface along x) check the steps there."""
    lb = library()
    R = 0.3 * n
    xi = int(n / 2 + R) - B // 2
    origins = [(xi, n // 2 - B // 2, z - B // 2) for z in cuts] + [(0, 0, cuts[0] - B // 2)]
    _check_boxes(lb, lb.D3Q19, (n, n, n), origins)
