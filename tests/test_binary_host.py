"""Host-side helpers of paper_0710_5470_gb300/binary.py against the binary oracle (no GPU)."""
import numpy as np

from oracle import binary_oracle as BO
from paper_0710_5470_gb300 import binary


def test_closed_forms_match_oracle():
    for A, B, k in ((-0.04, 0.04, 0.08), (-0.1, 0.2, 0.05)):
        assert abs(binary.phi_star(A, B) - BO.phi_star(A, B)) < 1e-15
        assert abs(binary.interface_width(A, k) - BO.interface_width(A, k)) < 1e-15
        assert abs(binary.surface_tension(A, B, k) / BO.surface_tension(A, B, k) - 1) < 1e-14


def test_drop_matches_oracle_drop():
    n, R = 40, 9.5
    A, B, k = -0.04, 0.04, 0.08
    want = BO.drop_phi((1, n, n), [(n / 2, n / 2)], [R], 1.0, -1.0, BO.interface_width(A, k))[0]
    assert np.abs(binary.drop_phi(n, R, A, k, B) - want).max() < 1e-14


def test_drop_3d_matches_oracle_drop():
    n, R = 20, 5.5
    A, B, k = -0.04, 0.04, 0.08
    want = BO.drop_phi((n, n, n), [(n / 2, n / 2, n / 2)], [R], 1.0, -1.0, BO.interface_width(A, k))
    assert np.abs(binary.drop_phi(n, R, A, k, B, dim=3) - want).max() < 1e-14
