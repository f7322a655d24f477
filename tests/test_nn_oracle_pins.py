"""Pins of the FP64 network oracle: brute force and SciPy for the
convolution, finite differences for every gradient, adjoint identities for
pooling and upsampling."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import nn


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv3d_brute_force():
    x = _rand((1, 3, 4, 5, 2), 0)
    w = _rand((3, 27, 2), 1)
    b = _rand(3, 2)
    y = nn.conv3d(x, w, b)
    N, D, H, W, C = x.shape
    for z in range(D):
        for yy in range(H):
            for xx in range(W):
                for co in range(3):
                    s = b[co]
                    for kz in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                zi, yi, xi = z + kz - 1, yy + ky - 1, xx + kx - 1
                                if 0 <= zi < D and 0 <= yi < H and 0 <= xi < W:
                                    s += w[co, kz * 9 + ky * 3 + kx] @ x[0, zi, yi, xi]
                    assert abs(y[0, z, yy, xx, co] - s) < 1e-12


def test_conv3d_equals_scipy_correlate():
    x = _rand((2, 6, 5, 7, 3), 3)
    w = _rand((4, 27, 3), 4)
    y = nn.conv3d(x, w)
    for n in range(2):
        for co in range(4):
            ref = sum(ndimage.correlate(x[n, ..., ci], w[co, :, ci].reshape(3, 3, 3), mode="constant", cval=0.0)
                      for ci in range(3))
            np.testing.assert_allclose(y[n, ..., co], ref, atol=1e-12)


def _fd(f, a, idx, h=1e-6):
    a1 = a.copy(); a1[idx] += h
    a2 = a.copy(); a2[idx] -= h
    return (f(a1) - f(a2)) / (2 * h)


def test_conv_gradients_by_finite_differences():
    x = _rand((1, 4, 4, 4, 3), 5)
    w = _rand((2, 27, 3), 6)
    b = _rand(2, 7)
    R = _rand((1, 4, 4, 4, 2), 8)
    L = lambda x_, w_, b_: float(np.sum(nn.conv3d(x_, w_, b_) * R))
    gx = nn.conv3d_dgrad(R, w)
    gw, gb = nn.conv3d_wgrad(R, x)
    rng = np.random.default_rng(9)
    for _ in range(10):
        i = tuple(rng.integers(0, s) for s in x.shape)
        assert abs(_fd(lambda a: L(a, w, b), x, i) - gx[i]) < 1e-6
        j = tuple(rng.integers(0, s) for s in w.shape)
        assert abs(_fd(lambda a: L(x, a, b), w, j) - gw[j]) < 1e-6
    for k in range(2):
        assert abs(_fd(lambda a: L(x, w, a), b, (k,)) - gb[k]) < 1e-6


def test_pool_and_upsample_adjoints():
    x = _rand((2, 4, 6, 4, 3), 10)
    y, arg = nn.maxpool2(x)
    # pooling picks the block maximum
    assert np.allclose(y[0, 1, 2, 1, 2], x[0, 2:4, 4:6, 2:4, 2].max())
    g = _rand(y.shape, 11)
    gx = nn.maxpool2_bwd(g, arg, x.shape)
    L = lambda a: float(np.sum(nn.maxpool2(a)[0] * g))
    rng = np.random.default_rng(12)
    for _ in range(10):
        i = tuple(rng.integers(0, s) for s in x.shape)
        assert abs(_fd(L, x, i) - gx[i]) < 1e-6
    u = _rand((1, 2, 3, 2, 4), 13)
    v = _rand((1, 4, 6, 4, 4), 14)
    assert abs(np.sum(nn.upsample2(u) * v) - np.sum(u * nn.upsample2_bwd(v))) < 1e-10


def test_mse_gradient():
    y, t = _rand((3, 4), 15), _rand((3, 4), 16)
    L, g = nn.mse(y, t)
    assert abs(L - np.mean((y - t) ** 2)) < 1e-14
    assert abs(_fd(lambda a: nn.mse(a, t)[0], y, (1, 2)) - g[1, 2]) < 1e-8


def test_unet_gradients_by_finite_differences():
    P = nn.init_params(seed=3, scale=0.7)
    for name, cin, cout in nn.LAYERS:
        w, b = P[name]
        P[name] = (w, np.random.default_rng(len(name)).normal(0, 0.05, cout) * (np.arange(cout) < (1 if name == "head" else cout)))
    x = np.zeros((1, 8, 8, 8, 16))
    x[..., :2] = _rand((1, 8, 8, 8, 2), 17)
    t = _rand((1, 8, 8, 8), 18)

    def loss(params):
        pred, _ = nn.unet_forward(x, params)
        return nn.mse(pred, t)[0]

    pred, cache = nn.unet_forward(x, P)
    _, gpred = nn.mse(pred, t)
    G = nn.unet_backward(gpred, cache, P)
    rng = np.random.default_rng(19)
    for name in ("e0a", "e1b", "b_b", "d2a", "d0a", "head"):
        w, b = P[name]
        for _ in range(3):
            j = tuple(rng.integers(0, s) for s in w.shape)
            if name == "head":
                j = (0,) + j[1:]
            fd = _fd(lambda a: loss({**P, name: (a, b)}), w, j, h=1e-5)
            assert abs(fd - G[name][0][j]) <= 1e-5 * max(1.0, abs(fd)), (name, j, fd, G[name][0][j])
        fdb = _fd(lambda a: loss({**P, name: (w, a)}), b, (0,), h=1e-5)
        assert abs(fdb - G[name][1][0]) <= 1e-5 * max(1.0, abs(fdb))
