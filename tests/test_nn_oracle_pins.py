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


# ---------------------------------------------------------------------------
# BF16 storage, Adam and the seeding transform
# ---------------------------------------------------------------------------
def test_bf16_rounding_is_nearest_with_ties_to_even():
    """Against the definition (the nearer of the two bfloat16 neighbours,
    ties to the even one) and against torch's float -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        np.float32(1.0) + np.arange(1, 200) * np.float32(2.0 ** -23)])   # includes exact ties
    x32 = x.astype(np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    lo = (bits & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)      # toward zero
    hi = ((bits & 0xFFFF0000) + 0x10000).astype(np.uint32).view(np.float32).astype(np.float64)
    v = x32.astype(np.float64)
    dlo, dhi = np.abs(v - lo), np.abs(hi - v)
    lo_even = ((bits >> 16) & 1) == 0
    want = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo_even, lo, hi)))
    got = nn.bf16(x)
    np.testing.assert_array_equal(got, want)
    ref = torch.from_numpy(x32).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, ref)
    # 8 significant bits: half an ulp is at most 2^-8 of the value
    assert (got != v).any() and (np.abs(got / v - 1) <= 2.0 ** -8).all()


def test_adam_first_step_moves_each_parameter_by_lr_times_sign():
    """From zero moments the bias corrections give m_hat = g and
    v_hat = g^2, so the first update is lr g / (|g| + eps)."""
    rng = np.random.default_rng(12)
    th = rng.standard_normal(500)
    g = rng.standard_normal(500) * 10.0 ** rng.integers(-3, 3, 500)
    t1, m1, v1 = nn.adam_step(th, g, np.zeros(500), np.zeros(500), 1, 1e-3)
    np.testing.assert_allclose(th - t1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)
    t0, _, _ = nn.adam_step(th, np.zeros(500), np.zeros(500), np.zeros(500), 1, 1e-3)
    np.testing.assert_array_equal(t0, th)


def test_adam_constant_gradient_moves_lr_every_step():
    """With the same gradient every step the bias-corrected moments stay
    g and g^2: k steps move by k lr g / (|g| + eps)."""
    g = np.array([3.0, -0.25, 1e-3, -40.0])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        th, m, v = nn.adam_step(th, g, m, v, t, 0.01)
    np.testing.assert_allclose(th, -7 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_adam_two_steps_closed_form():
    """Two steps with g1 then g2, worked out by hand: m_hat2 = (b1 g1 + g2) /
    (1 + b1), v_hat2 = (b2 g1^2 + g2^2) / (1 + b2)."""
    rng = np.random.default_rng(13)
    g1, g2 = rng.standard_normal(300), rng.standard_normal(300)
    th0 = rng.standard_normal(300)
    b1, b2, lr, eps = 0.9, 0.999, 2e-3, 1e-8
    th1, m, v = nn.adam_step(th0, g1, np.zeros(300), np.zeros(300), 1, lr)
    th2, m, v = nn.adam_step(th1, g2, m, v, 2, lr)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 * g1 + g2 * g2) / (1 + b2)
    step1 = lr * g1 / (np.abs(g1) + eps)
    np.testing.assert_allclose(th2, th0 - step1 - lr * mh / (np.sqrt(vh) + eps), rtol=1e-11, atol=1e-14)


def test_seed_transform_closed_forms():
    rng = np.random.default_rng(14)
    T1 = rng.uniform(3.0, 500.0, 1000)
    # zero prediction: T1 exp(y_mean)
    np.testing.assert_allclose(nn.seed_transform(T1, np.zeros(1000), 0.0, 1.0), T1, rtol=1e-15)
    np.testing.assert_allclose(nn.seed_transform(T1, np.zeros(1000), 0.3, 2.0), np.clip(T1 * np.exp(0.3), 2.7, 3000),
                               rtol=1e-15)
    # the prediction of the normalised ln T - ln T1 returns T
    T = rng.uniform(3.0, 2000.0, 1000)
    ym, ys = 0.12, 0.4
    p = (np.log(T) - np.log(T1) - ym) / ys
    np.testing.assert_allclose(nn.seed_transform(T1, p, ym, ys), T, rtol=1e-12)
    # clamps
    assert nn.seed_transform([100.0], [1e3], 0.0, 1.0)[0] == 3000.0
    assert nn.seed_transform([100.0], [-1e3], 0.0, 1.0)[0] == 2.7


def test_seed_transform_shrink_and_envelope_by_hand():
    """Two bins over ln T1 in [0, 2): bin 0 bounds y to [0.1, 0.5], bin 1 to
    [0, 0.2]; T1 below the range uses bin 0, above it bin 1."""
    env = (0.0, 2.0, [0.1, 0.0], [0.5, 0.2])
    T1 = np.array([3.0, 3.0, 3.0, 5.0, 5.0, 100.0])
    pred = np.array([0.0, 2.0, -3.0, 0.15, 3.0, 0.3])
    got = nn.seed_transform(T1, pred, 0.0, 1.0, envelope=env)
    # ln 3 = 1.0986 -> bin 1; ln 5 = 1.609 -> bin 1; ln 100 = 4.6 -> bin 1 (extended)
    want_y = np.array([0.0, 0.2, 0.0, 0.15, 0.2, 0.2])
    np.testing.assert_allclose(got, T1 * np.exp(want_y), rtol=1e-15)
    env2 = (1.2, 3.0, [0.1, 0.0], [0.5, 0.2])                 # ln 3 below the range -> bin 0
    np.testing.assert_allclose(nn.seed_transform([3.0, 3.0], [0.0, 2.0], 0.0, 1.0, envelope=env2),
                               3.0 * np.exp([0.1, 0.5]), rtol=1e-15)
    # shrink multiplies the de-normalised prediction before the bounds
    np.testing.assert_allclose(nn.seed_transform([10.0], [1.0], 0.5, 2.0, shrink=0.25), 10.0 * np.exp(0.625),
                               rtol=1e-15)


def test_seed_features_standardise_their_own_statistics():
    rng = np.random.default_rng(15)
    T1 = rng.uniform(5.0, 300.0, 4096)
    rho = np.exp(rng.normal(0.0, 1.5, 4096))
    lt, lr = np.log(T1), np.log(rho)
    norm = dict(lt_mean=lt.mean(), lt_std=lt.std(), lr_mean=lr.mean(), lr_std=lr.std())
    x = nn.seed_features(T1, rho, norm)
    np.testing.assert_allclose(x.mean(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(x.std(axis=0), 1.0, rtol=1e-12)
    # the third feature is the standardised change of ln T
    Tp = T1 * rng.uniform(0.5, 1.0, T1.size)
    d = np.log(T1) - np.log(Tp)
    x3 = nn.seed_features(T1, rho, dict(norm, ld_mean=d.mean(), ld_std=d.std()), T_prev=Tp)
    np.testing.assert_allclose(x3[:, :2], x, rtol=1e-15)
    np.testing.assert_allclose(x3[:, 2], (d - d.mean()) / d.std(), rtol=1e-12, atol=1e-12)
    # the fourth is the standardised change one iteration earlier (T_prev to
    # T_prev2), the first three as with three features (temperatures kept
    # above the 2.7 K clamp)
    Ta = rng.uniform(20.0, 300.0, 4096)
    Tb = Ta * rng.uniform(0.5, 1.0, Ta.size)
    Tc = Tb * rng.uniform(0.5, 1.0, Ta.size)
    da, e = np.log(Ta) - np.log(Tb), np.log(Tb) - np.log(Tc)
    n3 = dict(norm, ld_mean=da.mean(), ld_std=da.std())
    x4 = nn.seed_features(Ta, rho, dict(n3, pd_mean=e.mean(), pd_std=e.std()), T_prev=Tb, T_prev2=Tc)
    assert x4.shape == (Ta.size, 4)
    np.testing.assert_allclose(x4[:, :3], nn.seed_features(Ta, rho, n3, T_prev=Tb), rtol=1e-15)
    np.testing.assert_allclose(x4[:, 3], (e - e.mean()) / e.std(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(x4[:, 3].std(), 1.0, rtol=1e-12)
    # identity normalisation gives the logarithms; T1 below 2.7 K and rho = 0 are clamped
    x0 = nn.seed_features([1.0, 10.0], [0.0, 2.0], dict(lt_mean=0.0, lt_std=1.0, lr_mean=-60.0, lr_std=20.0))
    np.testing.assert_allclose(x0, [[np.log(2.7), (np.log(1e-30) + 60) / 20], [np.log(10.0), (np.log(2.0) + 60) / 20]],
                               rtol=1e-15)
    # standardised values beyond 6 are clipped
    xc = nn.seed_features([3000.0, 2.7, 90.0], [1.0] * 3, dict(lt_mean=4.5, lt_std=0.5, lr_mean=0.0, lr_std=1.0))
    np.testing.assert_allclose(xc[:, 0], [6.0, -6.0, (np.log(90.0) - 4.5) / 0.5], rtol=1e-15)


def test_bf16_storage_rounds_every_stored_tensor_and_nothing_else():
    """With BF16 storage every stored hidden activation is a bfloat16 value
    and the head output is not rounded; the result stays near the unrounded
    network (prediction within a few roundings; weight gradients within 20 %
    at the first layer, the end of the longest chain of roundings, and 2 %
    at the head)."""
    rng = np.random.default_rng(16)
    P = nn.init_params(seed=3)
    for n, _, cout in nn.LAYERS:
        P[n] = (P[n][0], rng.normal(0, 0.05, cout))
    x = np.zeros((1, 8, 8, 8, 16))
    x[..., :2] = rng.standard_normal((1, 8, 8, 8, 2))
    p0, a0 = nn.unet_forward(x, P)
    p1, a1 = nn.unet_forward(x, P, store_bf16=True)
    rel = np.linalg.norm(p1 - p0) / np.linalg.norm(p0)
    assert 1e-4 < rel < 3e-2
    for n, _, _ in nn.LAYERS[:-1]:
        assert np.array_equal(a1[n], nn.bf16(a1[n])), n
    assert not np.array_equal(a1["head"], nn.bf16(a1["head"]))
    g = rng.standard_normal(p0.shape)
    G0 = nn.unet_backward(g, a0, P)
    G1 = nn.unet_backward(g, a1, P, store_bf16=True)
    for n, _, _ in nn.LAYERS:
        r = np.linalg.norm(G1[n][0] - G0[n][0]) / np.linalg.norm(G0[n][0])
        assert r < (2e-2 if n == "head" else 0.2), (n, r)
