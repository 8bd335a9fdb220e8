"""Warm-start network kernels (lb_ws_*) against the numpy oracle.

Weights are fp16 on the GPU; the oracle runs in float64 with the same
fp16-rounded weights, so the comparison isolates the kernels' float32
arithmetic: outputs within 1e-3 and gradients within 1e-2 relative (norm of
each parameter block), the tolerances stated for the fp16-weight network.
"""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from tests.helpers import library

pytestmark = pytest.mark.gpu

CHANNELS = [5, 32, 32, 32, 3]


def _packed(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def _as_fp16_params(params):
    out = []
    for W, b in params:
        out.append((W.astype(np.float16).astype(np.float64), b.astype(np.float32).astype(np.float64)))
    return out


def _unpack(vec, like):
    out, o = [], 0
    for W, b in like:
        out.append((vec[o:o + W.size].reshape(W.shape), vec[o + W.size:o + W.size + b.size]))
        o += W.size + b.size
    return out


def test_forward_matches_oracle():
    lb = library()
    rng = np.random.default_rng(0)
    params = C.init_params(CHANNELS, seed=1)
    params = [(W, rng.uniform(-0.1, 0.1, b.shape)) for W, b in params]
    x = rng.uniform(-1, 1, (2, 5, 24, 37))
    with lb.WarmStart() as ws:
        ws.set_params(_packed(params))
        y = ws.forward(x.astype(np.float32))
    want, _ = C.forward(x.astype(np.float32).astype(np.float64), _as_fp16_params(params))
    assert np.abs(y - want).max() <= 1e-3 * np.abs(want).max()


def test_gradients_match_oracle():
    lb = library()
    rng = np.random.default_rng(2)
    params = C.init_params(CHANNELS, seed=3)
    params = [(W * 2.0, rng.uniform(-0.1, 0.1, b.shape)) for W, b in params]
    x = rng.uniform(-1, 1, (3, 5, 20, 18)).astype(np.float32)
    t = rng.uniform(-1, 1, (3, 3, 20, 18)).astype(np.float32)
    with lb.WarmStart() as ws:
        ws.set_params(_packed(params))
        loss, g = ws.loss_grad(x, t)
    p16 = _as_fp16_params(params)
    want_loss, want = C.loss_and_grads(x.astype(np.float64), t.astype(np.float64), p16)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    got = _unpack(g.astype(np.float64), params)
    for (dW, db), (wW, wb) in zip(got, want):
        assert np.linalg.norm(dW - wW) <= 1e-2 * np.linalg.norm(wW)
        assert np.linalg.norm(db - wb) <= 1e-2 * np.linalg.norm(wb) + 1e-7


def test_training_reduces_loss_on_a_smooth_target():
    """A learnable map (a smooth function of the input planes) is fitted."""
    lb = library()
    rng = np.random.default_rng(5)
    n, H, W = 32, 16, 16
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    x = np.zeros((n, 5, H, W), dtype=np.float32)
    t = np.zeros((n, 3, H, W), dtype=np.float32)
    for k in range(n):
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.uniform(-1, 1)
        x[k, 0] = np.sin(2 * np.pi * xx / W + ph)
        x[k, 1] = a
        t[k, 0] = 0.5 * np.sin(2 * np.pi * xx / W + ph) * a
        t[k, 1] = np.cos(2 * np.pi * xx / W + ph) * 0.3
    with lb.WarmStart(seed=7) as ws:
        hist = ws.train(x, t, epochs=60, batch=8, lr=1e-2)
    assert hist[-1] < 0.1 * hist[0], hist
