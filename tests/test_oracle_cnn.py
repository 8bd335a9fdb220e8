"""Pins of the warm-start network oracle: the periodic convolution against a
direct loop definition, translation equivariance, and backpropagation
against central finite differences (float64, relative 1e-6)."""
import numpy as np

from oracle import cnn_oracle as C


def _direct_conv(h, W, b):
    N, Cin, H, Wd = h.shape
    out = np.zeros((N, W.shape[0], H, Wd))
    for n in range(N):
        for o in range(W.shape[0]):
            for y in range(H):
                for x in range(Wd):
                    acc = b[o]
                    for c in range(Cin):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                acc += W[o, c, dy + 1, dx + 1] * h[n, c, (y + dy) % H, (x + dx) % Wd]
                    out[n, o, y, x] = acc
    return out


def test_conv_matches_direct_definition():
    rng = np.random.default_rng(0)
    h = rng.standard_normal((2, 3, 5, 4))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    assert np.allclose(C.conv3x3(h, W, b), _direct_conv(h, W, b), rtol=1e-13, atol=1e-13)


def test_conv_is_translation_equivariant():
    rng = np.random.default_rng(1)
    h = rng.standard_normal((1, 4, 7, 6))
    W = rng.standard_normal((3, 4, 3, 3))
    b = rng.standard_normal(3)
    a = C.conv3x3(np.roll(h, (2, -1), axis=(2, 3)), W, b)
    assert np.allclose(a, np.roll(C.conv3x3(h, W, b), (2, -1), axis=(2, 3)), atol=1e-13)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = C.init_params([2, 3, 3, 2], seed=4)
    params = [(W * 3.0, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((2, 2, 6, 5))
    t = rng.standard_normal((2, 2, 6, 5))
    loss, grads = C.loss_and_grads(x, t, params)
    eps = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = C.loss_and_grads(x, t, params)
                flat[idx] = old - eps
                lm, _ = C.loss_and_grads(x, t, params)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1e-3, abs(fd)), (li, idx, fd, g.reshape(-1)[idx])


def test_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    h = rng.standard_normal((1, 2, 4, 5))
    W = rng.standard_normal((3, 2, 3, 3))
    b = np.zeros(3)
    dout = rng.standard_normal((1, 3, 4, 5))
    dh, dW, db = C.conv3x3_backward(h, W, dout)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 3, 4), (0, 1, 2, 2)]:
        hp = h.copy(); hp[idx] += eps
        hm = h.copy(); hm[idx] -= eps
        fd = (np.sum(dout * C.conv3x3(hp, W, b)) - np.sum(dout * C.conv3x3(hm, W, b))) / (2 * eps)
        assert abs(fd - dh[idx]) < 1e-7 * max(1.0, abs(fd))
    assert np.allclose(db, dout.sum(axis=(0, 2, 3)))


# ---------------------------------------------------------------- 3D variant

def _direct_conv3(h, W, b):
    N, Cin, D, H, Wd = h.shape
    out = np.zeros((N, W.shape[0], D, H, Wd))
    for n in range(N):
        for o in range(W.shape[0]):
            for z in range(D):
                for y in range(H):
                    for x in range(Wd):
                        acc = b[o]
                        for c in range(Cin):
                            for dz in (-1, 0, 1):
                                for dy in (-1, 0, 1):
                                    for dx in (-1, 0, 1):
                                        acc += W[o, c, dz + 1, dy + 1, dx + 1] * \
                                            h[n, c, (z + dz) % D, (y + dy) % H, (x + dx) % Wd]
                        out[n, o, z, y, x] = acc
    return out


def test_conv3_matches_direct_definition():
    rng = np.random.default_rng(10)
    h = rng.standard_normal((1, 2, 3, 4, 5))
    W = rng.standard_normal((2, 2, 3, 3, 3))
    b = rng.standard_normal(2)
    assert np.allclose(C.conv3x3x3(h, W, b), _direct_conv3(h, W, b), rtol=1e-13, atol=1e-12)


def test_conv3_reduces_to_2d_on_a_one_plane_kernel():
    """A 3x3x3 kernel that is zero off the middle z slice is the 2D convolution of each plane."""
    rng = np.random.default_rng(11)
    h = rng.standard_normal((2, 3, 4, 5, 6))
    W2 = rng.standard_normal((2, 3, 3, 3))
    W3 = np.zeros((2, 3, 3, 3, 3))
    W3[:, :, 1] = W2
    b = rng.standard_normal(2)
    want = np.stack([C.conv3x3(h[:, :, z], W2, b) for z in range(h.shape[2])], axis=2)
    assert np.allclose(C.conv3x3x3(h, W3, b), want, atol=1e-13)


def test_backprop3_matches_finite_differences():
    rng = np.random.default_rng(12)
    params = C.init_params3([2, 3, 2], seed=5)
    params = [(W * 3.0, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((1, 2, 3, 4, 5))
    t = rng.standard_normal((1, 2, 3, 4, 5))
    loss, grads = C.loss_and_grads3(x, t, params)
    eps = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = C.loss_and_grads3(x, t, params)
                flat[idx] = old - eps
                lm, _ = C.loss_and_grads3(x, t, params)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1e-3, abs(fd)), (li, idx, fd, g.reshape(-1)[idx])
