"""Host steps of the learned warm start (no GPU): the network's input planes
and the decoding of a prediction into a start (rho, u) that keeps the tanh
start's mass, in 2D and 3D."""
import numpy as np
import pytest

from tests.helpers import library

RL, RG = 4.9, 2.2


def _tanh_start(shape, R, w=2.0):
    grids = np.meshgrid(*(np.arange(n) - n / 2 for n in shape), indexing="ij")
    d = np.sqrt(sum(g * g for g in grids))
    return RG + (RL - RG) * 0.5 * (1 + np.tanh((R - d) / w))


def test_features_planes():
    lb = library()
    r = _tanh_start((20, 24), 6.0)
    x = lb.ws_features(r, RL, RG, 0.55, 0.01, 0.9, 6.0)
    assert x.shape == (5, 20, 24) and x.dtype == np.float32
    assert np.allclose(x[0], (r - 0.5 * (RL + RG)) / (RL - RG), atol=1e-6)
    for c, v in zip(range(1, 5), ((0.55 - 0.53) / 0.03, (0.01 - 0.016) / 0.014, (0.9 - 1.05) / 0.45, 10.0 / 6.0)):
        assert np.allclose(x[c], v, atol=1e-6)


@pytest.mark.parametrize("shape", [(20, 24), (10, 12, 14)])
def test_decode_keeps_mass_and_scales_velocity(shape):
    lb = library()
    r = _tanh_start(shape, 0.3 * min(shape))
    rng = np.random.Generator(np.random.PCG64(5))
    y = rng.normal(0.0, 0.05, size=(len(shape) + 1,) + shape).astype(np.float32)
    decode = lb.ws_decode if len(shape) == 2 else lb.ws3_decode
    rho, u = decode(r, RL, RG, y)
    assert rho.sum() == pytest.approx(r.sum(), rel=1e-12)
    assert np.abs(rho - r).max() > 1e-3                      # the correction is applied
    assert np.allclose(u, 1e-3 * y[1:].astype(np.float64), rtol=0, atol=1e-12)
    rho0, u0 = decode(r, RL, RG, np.zeros_like(y))
    assert np.array_equal(rho0, r) and not u0.any()


def test_decode_rejects_bad_arguments():
    lb = library()
    r = _tanh_start((8, 8), 2.0)
    with pytest.raises(lb.LBError):
        lb.ws_decode(r, RG, RL, np.zeros((3, 8, 8), np.float32))     # rho_l <= rho_g
    with pytest.raises(lb.LBError):
        lb.ws_features(r, RL, RG, 0.55, 0.01, 0.9, 0.0)                # R <= 0
