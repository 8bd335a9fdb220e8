"""Host-side pieces of the scan module (no GPU)."""
import math

import pytest


def test_S_is_the_series_of_eq26():
    from paper_0710_5470_gb300 import scans
    for tau in (0.6, 0.789, 1.0, 1.5, 3.0):
        z = 1 - 1 / tau
        series = sum(i ** 3 * z ** (i - 1) for i in range(1, 4000)) / tau
        assert scans.S(tau) == pytest.approx(series, rel=1e-12, abs=1e-12)
    t0 = 0.5 + 0.5 / math.sqrt(3)
    assert abs(scans.S(t0)) < 1e-14 and scans.S(1.0) == 1.0


def test_flow_pattern_counts_the_vortex_ring():
    """flow_pattern on synthetic rings of 2m vortices (stream function
    g(r) sin(m theta) around a centred drop): the radial velocity on the
    probe circle changes sign 2m times and mode m dominates."""
    import numpy as np
    from paper_0710_5470_gb300 import scans
    n = 100
    y, x = np.mgrid[0:n, 0:n]
    X, Y = x - n / 2, y - n / 2
    r, th = np.hypot(X, Y), np.arctan2(Y, X)
    rho = np.where(r < 25, 4.5, 2.5)
    for m in (2, 4, 6):
        psi = np.exp(-((r - 33) / 10) ** 2) * np.sin(m * th) * 1e-5
        ux = 0.5 * (np.roll(psi, -1, 0) - np.roll(psi, 1, 0))
        uy = -0.5 * (np.roll(psi, -1, 1) - np.roll(psi, 1, 1))
        res = scans.flow_pattern(rho, np.stack([ux, uy]), 4.5, 2.5)
        assert res["ur_sign_changes"] == 2 * m
        assert res["dominant_mode"] == m
        assert abs(res["R_e"] - 25) < 0.5
