"""Host logic of the D3Q19 step's CTA work list (lb_work_list, no GPU).

For many lattice shapes, SM counts and occupancies: the (tile, z chunk) items
cover every column tile's planes exactly once, chunks are non-empty and at
least 4 planes long where the lattice allows, CTAs are listed longest chunk
first, small lattices fill exactly the resident slots, and lattices with fewer
than two slots per tile give every tile the same number of chunks.  The GB300
choices measured for 224^3, 256^3 and 320^3 are pinned.
"""
import itertools

import numpy as np
import pytest

from tests.helpers import library


def _check(w, shape, tile, sms, occ):
    nx, ny, nz = shape
    gx, gy = -(-nx // tile[0]), -(-ny // tile[1])
    assert len(w) > 0
    cover = {}
    for x0, y0, z0, z1 in w:
        assert x0 % tile[0] == 0 and y0 % tile[1] == 0 and 0 <= x0 < nx and 0 <= y0 < ny
        assert 0 <= z0 < z1 <= nz
        cover.setdefault((x0, y0), []).append((z0, z1))
    assert len(cover) == gx * gy
    for chunks in cover.values():
        chunks.sort()
        assert chunks[0][0] == 0 and chunks[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(chunks, chunks[1:]))
        if nz >= 4:
            assert min(z1 - z0 for z0, z1 in chunks) >= 4 or len(chunks) == 1
    lengths = w[:, 3] - w[:, 2]
    assert np.all(lengths[:-1] >= lengths[1:])
    tiles, slots = gx * gy, sms * occ
    per_tile = [len(c) for c in cover.values()]
    if 2 * tiles > slots:
        assert len(set(per_tile)) == 1
    elif all(n < max(1, nz // 4) for n in per_tile):
        assert len(w) == slots


SHAPES = [(1, 1, 1), (2, 3, 5), (32, 8, 4), (40, 24, 16), (33, 9, 7), (64, 64, 64), (96, 96, 96), (128, 128, 128),
          (192, 192, 192), (224, 224, 224), (256, 256, 256), (320, 320, 320), (512, 512, 512), (130, 70, 250),
          (1024, 1024, 1024), (2048, 16, 3)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_work_list_partitions_the_lattice(shape):
    lb = library()
    for sms, occ, tile in itertools.product((1, 7, 152), (1, 2, 3), ((32, 8), (32, 4))):
        _check(lb.work_list(sms, occ, shape, tile), shape, tile, sms, occ)


def test_work_list_gb300_choices():
    """The choices for a GB300 (152 SMs) and 32 x 8 tiles: the one-wave fill at
    128^3, and the number of z chunks per tile of the larger cubes, for the
    tile kernel (2 resident CTAs per SM) and the pair kernel (3).  Measured
    with the wave model that counts resident CTAs (fp16 pair kernel, GLUPS,
    against the model that did not): 256^3 33.9 (32.6), 384^3 35.4 (32.2),
    512^3 37.4 (34.9), 320^3 35.3 (36.3); float32 tile kernel within 1%."""
    lb = library()
    w = lb.work_list(152, 2, (128, 128, 128))
    assert len(w) == 304 and sorted(set((w[:, 3] - w[:, 2]).tolist())) == [25, 26, 32]
    w = lb.work_list(152, 3, (128, 128, 128))
    assert len(w) == 456 and sorted(set((w[:, 3] - w[:, 2]).tolist())) == [16, 18, 19]
    for occ, n, c in ((2, 224, 3), (2, 256, 7), (2, 320, 3), (2, 1024, 2),
                      (3, 256, 5), (3, 320, 9), (3, 384, 3), (3, 512, 4), (3, 1024, 1)):
        w = lb.work_list(152, occ, (n, n, n))
        assert len(w) == c * (-(-n // 32)) * (-(-n // 8)), (occ, n)


def test_work_list_rejects_bad_sizes():
    lb = library()
    for args in ((0, 2, (8, 8, 8)), (152, 0, (8, 8, 8)), (152, 2, (0, 8, 8)), (152, 2, (1300, 1300, 1300))):
        with pytest.raises(lb.LBError):
            lb.work_list(*args)
