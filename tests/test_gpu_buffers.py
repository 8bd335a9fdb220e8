"""lb_create_with_buffers: a context on caller-owned device memory (a torch
allocation) steps bit for bit like one on its own allocation, keeps its
populations in that memory, and leaves it to the caller on destroy."""
import numpy as np
import pytest

from tests.helpers import A_VDW, B_VDW, library

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lat, shape, storage", [(0, (40, 24), 2), (0, (33, 17), 1), (1, (64, 12, 10), 2),
                                                 (1, (20, 12, 9), 0), (1, (32, 8, 6), 3)])
def test_caller_buffer_matches_own_allocation(lat, shape, storage):
    import torch
    lb = library()
    args = (lat, shape, A_VDW, B_VDW, 0.55, 0.01, 1.0)
    kw = dict(scheme=lb.FORCING, storage=storage)
    need = lb.population_bytes(*args, **kw)
    buf = torch.zeros(need + 512, dtype=torch.uint8, device="cuda")[:need]
    assert buf.data_ptr() % 256 == 0
    centre = [tuple(n / 2 for n in shape)]
    out = []
    for b in (None, buf):
        with lb.Context(*args, **kw, buffer=b) as ctx:
            ctx.init_drops(centre, [0.3 * min(shape)], 2.0)
            ctx.step(50)
            out.append(ctx.get_populations())
            if b is not None:
                ptr, nbytes = ctx.device_state()
                assert buf.data_ptr() <= ptr < buf.data_ptr() + need   # the current buffer lives in it
    assert np.array_equal(out[0], out[1])
    torch.cuda.synchronize()
    assert int(buf.count_nonzero()) > 0      # still the caller's, after destroy
