"""Host logic of the time-to-steady driver (no GPU): the drop centre on the
periodic lattice, the accuracy comparison and the sweep summary."""
import numpy as np
import pytest

from paper_0710_5470_gb300 import steady


def _drop(nx, ny, cx, cy, R=8.0, w=2.0):
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    dx = (x - cx + nx / 2) % nx - nx / 2
    dy = (y - cy + ny / 2) % ny - ny / 2
    return 1.0 + 3.0 * 0.5 * (1 + np.tanh((R - np.hypot(dx, dy)) / w))


@pytest.mark.parametrize("cx,cy", [(20.0, 16.0), (3.0, 30.0), (47.5, 0.5), (0.0, 0.0)])
def test_centre_of_a_drop_across_the_periodic_boundary(cx, cy):
    c = steady._centre(_drop(48, 36, cx, cy))
    d = (c - np.array([cx, cy]) + np.array([24, 18])) % np.array([48, 36]) - np.array([24, 18])
    assert np.abs(d).max() < 1e-6


def test_compare_reports_shift_and_errors():
    r0 = _drop(48, 36, 20.0, 16.0)
    r1 = _drop(48, 36, 22.0, 16.0) * (1 + 1e-4)
    u0 = np.zeros((2, 36, 48))
    u0[0, 10, 10] = 2e-3
    u1 = u0 * 1.03
    ref = {"final": [(r0, u0), (r0, u0)], "status": [0, 4]}
    run = {"final": [(r1, u1), (r1, u1)], "status": [0, 0]}
    out = steady.compare(ref, run)
    assert out[1] is None
    c = out[0]
    assert abs(c["shift"] - 2.0) < 1e-6
    assert abs(c["max_u_rel_err"] - 0.03) < 1e-12
    assert abs(c["rho_max_err"] - r0.max() * 1e-4) < 1e-9


def test_sweep_summary_counts_and_updates():
    res = {"seconds": 2.0, "status": [0, 4, 5, 0], "steps": [100, 40, -1, 300], "batch_steps": 500}
    s = steady._sweep_summary(res, [10, 20, 30, 40])
    assert (s["converged"], s["unstable"], s["not_converged"], s["instances"]) == (2, 1, 1, 4)
    assert s["lattice_updates"] == 100 * 10 + 40 * 20 + 500 * 30 + 300 * 40   # capped: the whole batch
    assert s["mean_steps_converged"] == 200.0
    assert s["mlups"] == pytest.approx(s["lattice_updates"] / 2.0 / 1e6)
