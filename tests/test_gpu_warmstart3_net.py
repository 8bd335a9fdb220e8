"""3D warm-start network kernels (lb_ws3_*) against the numpy oracle.

As for the 2D network: fp16 weights on the GPU, the oracle in float64 with the
same fp16-rounded weights; outputs within 1e-3 and gradients within 1e-2
relative (norm of each parameter block).  Volumes are ragged against the
16 x 16 tiles and include a one-plane-deep case (periodic z wrap onto itself).
"""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from tests.helpers import library

pytestmark = pytest.mark.gpu

CHANNELS = [5, 32, 32, 32, 4]


def _packed(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def _as_fp16_params(params):
    return [(W.astype(np.float16).astype(np.float64), b.astype(np.float32).astype(np.float64)) for W, b in params]


def _unpack(vec, like):
    out, o = [], 0
    for W, b in like:
        out.append((vec[o:o + W.size].reshape(W.shape), vec[o + W.size:o + W.size + b.size]))
        o += W.size + b.size
    return out


@pytest.mark.parametrize("shape", [(2, 5, 6, 7), (1, 1, 17, 9), (1, 3, 20, 33)])
def test_forward3_matches_oracle(shape):
    lb = library()
    rng = np.random.default_rng(0)
    params = C.init_params3(CHANNELS, seed=1)
    params = [(W, rng.uniform(-0.1, 0.1, b.shape)) for W, b in params]
    n, D, H, W = shape
    x = rng.uniform(-1, 1, (n, 5, D, H, W))
    with lb.WarmStart3() as ws:
        assert ws.num_params == sum(Wt.size + b.size for Wt, b in params)
        ws.set_params(_packed(params))
        y = ws.forward(x.astype(np.float32))
    want, _ = C.forward3(x.astype(np.float32).astype(np.float64), _as_fp16_params(params))
    assert np.abs(y - want).max() <= 1e-3 * np.abs(want).max()


def test_gradients3_match_oracle():
    lb = library()
    rng = np.random.default_rng(2)
    params = C.init_params3(CHANNELS, seed=3)
    params = [(W * 2.0, rng.uniform(-0.1, 0.1, b.shape)) for W, b in params]
    x = rng.uniform(-1, 1, (2, 5, 4, 10, 9)).astype(np.float32)
    t = rng.uniform(-1, 1, (2, 4, 4, 10, 9)).astype(np.float32)
    with lb.WarmStart3() as ws:
        ws.set_params(_packed(params))
        loss, g = ws.loss_grad(x, t)
    p16 = _as_fp16_params(params)
    want_loss, want = C.loss_and_grads3(x.astype(np.float64), t.astype(np.float64), p16)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    got = _unpack(g.astype(np.float64), params)
    for (dW, db), (wW, wb) in zip(got, want):
        assert np.linalg.norm(dW - wW) <= 1e-2 * np.linalg.norm(wW)
        assert np.linalg.norm(db - wb) <= 1e-2 * np.linalg.norm(wb) + 1e-7


def test_training3_reduces_loss_on_a_smooth_target():
    lb = library()
    rng = np.random.default_rng(5)
    n, D, H, W = 16, 8, 8, 8
    zz, yy, xx = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    x = np.zeros((n, 5, D, H, W), dtype=np.float32)
    t = np.zeros((n, 4, D, H, W), dtype=np.float32)
    for k in range(n):
        ph, a = rng.uniform(0, 2 * np.pi), rng.uniform(-1, 1)
        x[k, 0] = np.sin(2 * np.pi * xx / W + ph) * np.cos(2 * np.pi * zz / D)
        x[k, 1] = a
        t[k, 0] = 0.5 * a * x[k, 0]
        t[k, 3] = 0.3 * np.tanh(x[k, 0])
    with lb.WarmStart3(seed=7) as ws:
        hist = ws.train(x, t, epochs=60, batch=4, lr=1e-2, seed=1)
    assert hist[-1] < 0.3 * hist[0]


def test_predict_sym3_is_reflection_symmetric():
    """A reflection-symmetric input gives a reflection-symmetric density and an odd velocity."""
    lb = library()
    D = H = W = 12
    zz, yy, xx = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    d = np.sqrt((xx - W / 2) ** 2 + (yy - H / 2) ** 2 + (zz - D / 2) ** 2)
    x = np.zeros((5, D, H, W), dtype=np.float32)
    x[0] = 0.5 * np.tanh((3.5 - d) / 2)
    x[1:] = 0.3
    with lb.WarmStart3(seed=3) as ws:
        y = ws.predict_sym(x)
    flip = lambda a, ax: np.roll(np.flip(a, axis=ax), 1, axis=ax)     # a -> (n - a) mod n
    assert np.allclose(y[0], flip(y[0], 2), atol=1e-6)                 # x reflection
    assert np.allclose(y[1], -flip(y[1], 2), atol=1e-6)                # u_x odd under it
    assert np.allclose(y[3], -flip(y[3], 0), atol=1e-6)                # u_z odd under z reflection
