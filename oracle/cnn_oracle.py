"""FP64 CPU oracle of the warm-start networks, 2D and 3D (test infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by tests/ (never by the CUDA product
path).  The warm start is a build addition, not part of the paper: a small
fully convolutional network maps (tanh-initialised density, T, kappa, tau, R)
planes to the steady density correction and velocity of a drop, so the
lattice Boltzmann run can start near its steady state.

Network: L layers of 3x3 convolutions with circular (periodic) padding,
  h_0 = x,  h_l = tanh(W_l * h_{l-1} + b_l) for l < L,  y = W_L * h_{L-1} + b_L,
W_l of shape (C_out, C_in, 3, 3) with (W * h)[o, y, x] =
  sum_{c, dy, dx} W[o, c, dy + 1, dx + 1] h[c, y + dy, x + dx]  (indices mod H, W).
Loss: mean squared error over all outputs of the batch.

Plain numpy, float64; the convolution is written as the sum over the nine
taps with np.roll.  Pinned by finite differences and by a direct loop
convolution in tests/test_oracle_cnn.py.
"""
from __future__ import annotations

import numpy as np


def conv3x3(h: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Periodic 3x3 convolution of h (N, C_in, H, W) -> (N, C_out, H, W)."""
    N, C, H, Wd = h.shape
    out = np.zeros((N, W.shape[0], H, Wd))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            # value at (y + dy, x + dx)
            sh = np.roll(h, shift=(-dy, -dx), axis=(2, 3))
            out += np.einsum("oc,ncyx->noyx", W[:, :, dy + 1, dx + 1], sh)
    return out + b[None, :, None, None]


def conv3x3_backward(h: np.ndarray, W: np.ndarray, dout: np.ndarray):
    """Gradients of sum(dout * conv3x3(h, W, b)) w.r.t. h, W and b."""
    dh = np.zeros_like(h)
    dW = np.zeros_like(W)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            sh = np.roll(h, shift=(-dy, -dx), axis=(2, 3))
            dW[:, :, dy + 1, dx + 1] = np.einsum("noyx,ncyx->oc", dout, sh)
            # out[y, x] reads h[y + dy, x + dx]: the gradient flows back shifted the other way
            contrib = np.einsum("oc,noyx->ncyx", W[:, :, dy + 1, dx + 1], dout)
            dh += np.roll(contrib, shift=(dy, dx), axis=(2, 3))
    db = dout.sum(axis=(0, 2, 3))
    return dh, dW, db


def forward(x: np.ndarray, params: list):
    """Network output and the per-layer activations (for the backward pass)."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv3x3(h, W, b)
        h = np.tanh(z) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grads(x: np.ndarray, target: np.ndarray, params: list):
    """MSE loss and its gradients (list of (dW, db)) by backpropagation."""
    y, acts = forward(x, params)
    n = y.size
    loss = float(np.sum((y - target) ** 2) / n)
    g = 2.0 * (y - target) / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        if li < len(params) - 1:
            g = g * (1.0 - acts[li + 1] ** 2)          # tanh'
        dh, dW, db = conv3x3_backward(acts[li], W, g)
        grads[li] = (dW, db)
        g = dh
    return loss, grads


def init_params(channels, seed: int = 0):
    """Layer parameters for channel counts e.g. [5, 32, 32, 32, 3]: W ~ U(-s, s)
    with s = 1/sqrt(9 C_in), b = 0 (numpy PCG64 seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        s = 1.0 / np.sqrt(9 * cin)
        params.append((rng.uniform(-s, s, (cout, cin, 3, 3)), np.zeros(cout)))
    return params


# --------------------------------------------------------------------------
# 3D variant: periodic 3x3x3 convolutions over (z, y, x), same layer pattern.
#   (W * h)[o, z, y, x] = sum_{c, dz, dy, dx} W[o, c, dz+1, dy+1, dx+1] h[c, z+dz, y+dy, x+dx]
# --------------------------------------------------------------------------

_TAPS3 = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3x3x3(h: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Periodic 3x3x3 convolution of h (N, C_in, D, H, W) -> (N, C_out, D, H, W)."""
    N, C, D, H, Wd = h.shape
    out = np.zeros((N, W.shape[0], D, H, Wd))
    for dz, dy, dx in _TAPS3:
        sh = np.roll(h, shift=(-dz, -dy, -dx), axis=(2, 3, 4))     # value at (z+dz, y+dy, x+dx)
        out += np.einsum("oc,nczyx->nozyx", W[:, :, dz + 1, dy + 1, dx + 1], sh)
    return out + b[None, :, None, None, None]


def conv3x3x3_backward(h: np.ndarray, W: np.ndarray, dout: np.ndarray):
    """Gradients of sum(dout * conv3x3x3(h, W, b)) w.r.t. h, W and b."""
    dh = np.zeros_like(h)
    dW = np.zeros_like(W)
    for dz, dy, dx in _TAPS3:
        sh = np.roll(h, shift=(-dz, -dy, -dx), axis=(2, 3, 4))
        dW[:, :, dz + 1, dy + 1, dx + 1] = np.einsum("nozyx,nczyx->oc", dout, sh)
        contrib = np.einsum("oc,nozyx->nczyx", W[:, :, dz + 1, dy + 1, dx + 1], dout)
        dh += np.roll(contrib, shift=(dz, dy, dx), axis=(2, 3, 4))
    db = dout.sum(axis=(0, 2, 3, 4))
    return dh, dW, db


def forward3(x: np.ndarray, params: list):
    """3D network output and per-layer activations."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv3x3x3(h, W, b)
        h = np.tanh(z) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grads3(x: np.ndarray, target: np.ndarray, params: list):
    """MSE loss and its gradients for the 3D network (backpropagation)."""
    y, acts = forward3(x, params)
    n = y.size
    loss = float(np.sum((y - target) ** 2) / n)
    g = 2.0 * (y - target) / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        if li < len(params) - 1:
            g = g * (1.0 - acts[li + 1] ** 2)
        dh, dW, db = conv3x3x3_backward(acts[li], W, g)
        grads[li] = (dW, db)
        g = dh
    return loss, grads


def init_params3(channels, seed: int = 0):
    """3D layer parameters: W ~ U(-s, s), s = 1/sqrt(27 C_in), b = 0 (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        s = 1.0 / np.sqrt(27 * cin)
        params.append((rng.uniform(-s, s, (cout, cin, 3, 3, 3)), np.zeros(cout)))
    return params
