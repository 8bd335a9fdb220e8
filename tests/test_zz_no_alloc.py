"""lb_field_stats_noalloc: float64 field reductions that allocate no device memory.

This entry point serves callers that cannot allocate device memory when they
need the numbers (their allocator already holds the memory they may use, or
their stepping loop must not pay for cudaMalloc/cudaFree synchronising the
device or risk an out-of-memory failure mid-run).  The caller passes device
fields and a device output buffer; the partial sums live in a fixed
file-scope device array of the library.  The test checks it through the C ABI
against lb_stats_get, within the float64 tolerance the other reduction tests
use, on two calls in a row of different sizes (so a call that read the
previous call's leftover partials would fail), and checks the size limit.
"""
import numpy as np
import pytest

from tests.helpers import library, make_ctx

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MAX_SITES = 4096 * 4096   # LB_NOALLOC_MAX_SITES of include/lb.h


def _device(a):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda")


def test_noalloc_stats_match_lb_stats_get_on_two_calls():
    lb = library()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    cases = [("D3Q19", "forcing", (24, 22, 20), 20), ("D2Q9", "equilibrium", (70, 50), 10)]
    for lat, scheme, shape, steps in cases:
        dim = 3 if lat == "D3Q19" else 2
        with make_ctx(lb, lat, scheme, shape) as ctx:
            centre = [s / 2.0 for s in shape]
            ctx.init_drops([centre], [0.3 * min(shape)])
            ctx.step(steps)
            want = ctx.stats()
            rho, u, v = ctx.fields()
        d_rho, d_u, d_v = _device(rho), _device(u), _device(v)
        n = rho.size
        out.fill_(float("nan"))
        lb.field_stats_noalloc(d_rho.data_ptr(), d_u.data_ptr(), d_v.data_ptr(), dim, n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert abs(got[0] - want["mass"]) <= 1e-12 * want["mass"]
        for c in range(dim):
            assert abs(got[1 + c] - want["momentum"][c]) <= 1e-12 * want["mass"]
        for c in range(dim, 3):
            assert got[1 + c] == 0.0
        assert abs(got[4] - want["max_u"]) <= 1e-15 + 1e-12 * want["max_u"]
        assert abs(got[5] - want["max_v"]) <= 1e-15 + 1e-12 * want["max_v"]
        assert got[6] == want["min_rho"] and got[7] == want["max_rho"]


def test_noalloc_rejects_sizes_beyond_its_array():
    lb = library()
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = small.data_ptr()
    with pytest.raises(lb.LBError) as e:
        lb.field_stats_noalloc(p, p, p, 3, MAX_SITES + 1, out.data_ptr())
    assert e.value.status == 1 and "exceeds the maximum" in str(e.value)
    with pytest.raises(lb.LBError):
        lb.field_stats_noalloc(p, p, p, 3, 0, out.data_ptr())
