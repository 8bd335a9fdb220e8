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


def test_symmetrize_is_exactly_symmetric_and_keeps_mass():
    """The predicted start is averaged over the symmetries fixing the box
    centre (mirrors x -> n - x, and axis permutations for equal sides) with
    every orbit summed in sorted order: mirror sites must be bitwise equal (a
    start symmetric only to rounding drives the drop off the centre), a
    symmetric field must come back unchanged to rounding, and the mass is kept."""
    import numpy as np
    from paper_0710_5470_gb300 import warmstart as W
    rng = np.random.default_rng(3)
    for shape in [(48, 48), (45, 45), (12, 10), (16, 16, 16), (9, 9, 9)]:
        a = rng.random(shape) + 2.0
        s = W.symmetrize(a)
        for ax in range(a.ndim):
            assert np.array_equal(W._reflect(s, ax), s)
        if len(set(shape)) == 1:
            assert np.array_equal(np.swapaxes(s, 0, 1), s)
        assert abs(s.sum() - a.sum()) <= 1e-13 * a.sum()
        assert np.allclose(W.symmetrize(s), s, rtol=1e-14, atol=0)     # an 8- or 48-term mean, rounded
    # a mirror about n/2 maps the centre site to itself and x to n - x
    x = np.arange(8.0)
    assert np.array_equal(W._reflect(x, 0), np.array([0, 7, 6, 5, 4, 3, 2, 1], dtype=float))


def test_spans_tells_a_drop_from_a_stripe():
    import numpy as np
    from paper_0710_5470_gb300 import warmstart as W
    rl, rg = 4.9, 2.2
    n = 40
    y, x = np.mgrid[0:n, 0:n]
    drop = np.where((x - 20) ** 2 + (y - 20) ** 2 < 12 ** 2, rl, rg)
    stripe = np.where(abs(y - 20) < 8, rl, rg)                 # liquid across x
    assert W.spans(drop, rl, rg) == [False, False]
    assert W.spans(stripe, rl, rg) == [True, False]
    z, y3, x3 = np.mgrid[0:16, 0:16, 0:16]
    cyl = np.where((x3 - 8) ** 2 + (y3 - 8) ** 2 < 25, rl, rg)  # liquid along z
    assert W.spans(cyl, rl, rg) == [False, False, True]
