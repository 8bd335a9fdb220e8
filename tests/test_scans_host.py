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
