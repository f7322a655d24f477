"""FP64 NumPy oracle of the learned temperature seed's network (test
infrastructure only; the CUDA path never imports it).

The method (paper Sect. 3.3-3.4, reference field and cheap early iterations)
has no network; this small 3D U-Net maps (log T after the first iteration,
log density) to the converged log T and seeds the Monte Carlo iteration.
Everything here is the plain definition in float64, channels-last
(N, D, H, W, C):

* conv3d: y[v, co] = b[co] + sum_{tap, ci} w[co, tap, ci] x[v + off(tap), ci],
  3x3x3 taps (tap = (kz*3 + ky)*3 + kx, offsets -1..1), zero padding 1;
* its gradients with respect to x, w and b (written out, and pinned by
  finite differences in the tests);
* 2x2x2 max pooling, nearest 2x upsampling, ReLU, mean squared error;
* the U-Net of four levels with channels 16-32-64-128 and skip concatenation
  [upsampled, skip], optionally with the BF16 storage of the network's stated
  precision (every stored activation and every layer's output gradient
  rounded to bfloat16, arithmetic in float64);
* one Adam step (Kingma & Ba 2015, Algorithm 1) on given parameters,
  gradients and moments;
* the seeding transform: the network input features from T after the first
  iteration and the density, and T_seed = T1 exp(prediction) with the
  prediction de-normalised.
"""
from __future__ import annotations

import numpy as np

TAPS = [(kz - 1, ky - 1, kx - 1) for kz in range(3) for ky in range(3) for kx in range(3)]


def _shift(x, dz, dy, dx):
    """x[v + (dz, dy, dx)] with zeros outside (x: N,D,H,W,C)."""
    N, D, H, W, C = x.shape
    out = np.zeros_like(x)
    zs = slice(max(0, -dz), D - max(0, dz)); zd = slice(max(0, dz), D - max(0, -dz) if dz < 0 else D)
    ys = slice(max(0, -dy), H - max(0, dy)); yd = slice(max(0, dy), H - max(0, -dy) if dy < 0 else H)
    xs = slice(max(0, -dx), W - max(0, dx)); xd = slice(max(0, dx), W - max(0, -dx) if dx < 0 else W)
    # out[z] = x[z + dz]
    out[:, zs, ys, xs, :] = x[:, zd, yd, xd, :]
    return out


def conv3d(x, w, b=None):
    """x (N,D,H,W,Cin), w (Cout, 27, Cin), b (Cout) -> (N,D,H,W,Cout)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:4] + (w.shape[0],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += np.tensordot(_shift(x, dz, dy, dx), w[:, t, :], axes=([4], [1]))
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_dgrad(gy, w):
    """dL/dx from dL/dy: gx[v, ci] = sum_{tap, co} w[co, tap, ci] gy[v - off(tap), co]."""
    gy = np.asarray(gy, np.float64)
    w = np.asarray(w, np.float64)
    gx = np.zeros(gy.shape[:4] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        gx += np.tensordot(_shift(gy, -dz, -dy, -dx), w[:, t, :], axes=([4], [0]))
    return gx


def conv3d_wgrad(gy, x):
    """dL/dw[co, tap, ci] = sum_v gy[v, co] x[v + off(tap), ci]; dL/db = sum_v gy."""
    gy = np.asarray(gy, np.float64)
    x = np.asarray(x, np.float64)
    gw = np.zeros((gy.shape[4], 27, x.shape[4]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shift(x, dz, dy, dx)
        gw[:, t, :] = np.tensordot(gy, xs, axes=([0, 1, 2, 3], [0, 1, 2, 3]))
    return gw, gy.sum(axis=(0, 1, 2, 3))


def bf16(x):
    """Round to the nearest bfloat16 (8 significant bits), ties to even, as
    a float64 array: the float32 value's bit pattern is rounded at bit 16
    (add 0x7fff plus the lowest kept bit, then drop the low 16 bits).
    Inputs are finite."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def relu(x):
    return np.maximum(x, 0.0)


def maxpool2(x):
    """2x2x2 max pooling; returns (y, argmax 0..7 = ox + 2 oy + 4 oz, first maximum)."""
    N, D, H, W, C = x.shape
    r = x.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C)
    r = r.transpose(0, 1, 3, 5, 2, 4, 6, 7).reshape(N, D // 2, H // 2, W // 2, 8, C)
    # octant order inside the 8: index = oz*4 + oy*2 + ox
    return r.max(axis=4), r.argmax(axis=4)


def maxpool2_bwd(gy, arg, shape):
    N, D, H, W, C = shape
    g8 = np.zeros((N, D // 2, H // 2, W // 2, 8, C))
    np.put_along_axis(g8, arg[:, :, :, :, None, :], gy[:, :, :, :, None, :], axis=4)
    g = g8.reshape(N, D // 2, H // 2, W // 2, 2, 2, 2, C).transpose(0, 1, 4, 2, 5, 3, 6, 7)
    return g.reshape(N, D, H, W, C)


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_bwd(gy):
    N, D, H, W, C = gy.shape
    return gy.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def mse(y, t):
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


# ---------------------------------------------------------------------------
# U-Net
# ---------------------------------------------------------------------------
# (name, input, output channels) in forward order; "cat" inputs are
# [upsampled deeper output, skip]
LAYERS = [("e0a", 16, 16), ("e0b", 16, 16), ("e1a", 16, 32), ("e1b", 32, 32),
          ("e2a", 32, 64), ("e2b", 64, 64), ("b_a", 64, 128), ("b_b", 128, 128),
          ("d2a", 192, 64), ("d2b", 64, 64), ("d1a", 96, 32), ("d1b", 32, 32),
          ("d0a", 48, 16), ("d0b", 16, 16), ("head", 16, 16)]


def unet_forward(x, params, store_bf16=False):
    """x (N,S,S,S,16) (2 real input channels, rest zero); params: name ->
    (w (Cout,27,Cin), b (Cout)).  Returns (prediction = head channel 0,
    cache of activations for the backward pass).  store_bf16: every hidden
    layer's output is stored as bfloat16 (the network's stated precision);
    the head stays unrounded."""
    P = params
    st = bf16 if store_bf16 else (lambda v: v)
    a = {}
    a["x"] = x
    a["e0a"] = st(relu(conv3d(x, *P["e0a"])))
    a["e0b"] = st(relu(conv3d(a["e0a"], *P["e0b"])))
    a["p0"], a["arg0"] = maxpool2(a["e0b"])
    a["e1a"] = st(relu(conv3d(a["p0"], *P["e1a"])))
    a["e1b"] = st(relu(conv3d(a["e1a"], *P["e1b"])))
    a["p1"], a["arg1"] = maxpool2(a["e1b"])
    a["e2a"] = st(relu(conv3d(a["p1"], *P["e2a"])))
    a["e2b"] = st(relu(conv3d(a["e2a"], *P["e2b"])))
    a["p2"], a["arg2"] = maxpool2(a["e2b"])
    a["b_a"] = st(relu(conv3d(a["p2"], *P["b_a"])))
    a["b_b"] = st(relu(conv3d(a["b_a"], *P["b_b"])))
    a["cat2"] = np.concatenate([upsample2(a["b_b"]), a["e2b"]], axis=4)
    a["d2a"] = st(relu(conv3d(a["cat2"], *P["d2a"])))
    a["d2b"] = st(relu(conv3d(a["d2a"], *P["d2b"])))
    a["cat1"] = np.concatenate([upsample2(a["d2b"]), a["e1b"]], axis=4)
    a["d1a"] = st(relu(conv3d(a["cat1"], *P["d1a"])))
    a["d1b"] = st(relu(conv3d(a["d1a"], *P["d1b"])))
    a["cat0"] = np.concatenate([upsample2(a["d1b"]), a["e0b"]], axis=4)
    a["d0a"] = st(relu(conv3d(a["cat0"], *P["d0a"])))
    a["d0b"] = st(relu(conv3d(a["d0a"], *P["d0b"])))
    a["head"] = conv3d(a["d0b"], *P["head"])
    return a["head"][..., 0], a


def unet_backward(g_pred, a, params, store_bf16=False):
    """Gradients of the loss (given dL/dprediction) for every parameter.
    store_bf16: each layer's output gradient (after its ReLU mask) is
    rounded to bfloat16 before it enters the weight, bias and input
    gradients of that layer (the network's stated precision)."""
    P = params
    G = {}
    gh = np.zeros(a["head"].shape)
    gh[..., 0] = g_pred
    st = bf16 if store_bf16 else (lambda v: v)

    def back(name, gy, x):
        gy = st(gy)
        G[name] = conv3d_wgrad(gy, x)
        return conv3d_dgrad(gy, P[name][0])

    g = back("head", gh, a["d0b"])
    g = back("d0b", g * (a["d0b"] > 0), a["d0a"])
    gcat0 = back("d0a", g * (a["d0a"] > 0), a["cat0"])
    c_up = a["d1b"].shape[4]
    g_d1b = upsample2_bwd(gcat0[..., :c_up])
    g_e0b = gcat0[..., c_up:]
    g = back("d1b", g_d1b * (a["d1b"] > 0), a["d1a"])
    gcat1 = back("d1a", g * (a["d1a"] > 0), a["cat1"])
    c_up = a["d2b"].shape[4]
    g_d2b = upsample2_bwd(gcat1[..., :c_up])
    g_e1b = gcat1[..., c_up:]
    g = back("d2b", g_d2b * (a["d2b"] > 0), a["d2a"])
    gcat2 = back("d2a", g * (a["d2a"] > 0), a["cat2"])
    c_up = a["b_b"].shape[4]
    g_bb = upsample2_bwd(gcat2[..., :c_up])
    g_e2b = gcat2[..., c_up:]
    g = back("b_b", g_bb * (a["b_b"] > 0), a["b_a"])
    g_p2 = back("b_a", g * (a["b_a"] > 0), a["p2"])
    g_e2b = g_e2b + maxpool2_bwd(g_p2, a["arg2"], a["e2b"].shape)
    g = back("e2b", g_e2b * (a["e2b"] > 0), a["e2a"])
    g_p1 = back("e2a", g * (a["e2a"] > 0), a["p1"])
    g_e1b = g_e1b + maxpool2_bwd(g_p1, a["arg1"], a["e1b"].shape)
    g = back("e1b", g_e1b * (a["e1b"] > 0), a["e1a"])
    g_p0 = back("e1a", g * (a["e1a"] > 0), a["p0"])
    g_e0b = g_e0b + maxpool2_bwd(g_p0, a["arg0"], a["e0b"].shape)
    g = back("e0b", g_e0b * (a["e0b"] > 0), a["e0a"])
    G["e0a"] = conv3d_wgrad(st(g * (a["e0a"] > 0)), a["x"])
    return G


# ---------------------------------------------------------------------------
# Adam (Kingma & Ba 2015, Algorithm 1)
# ---------------------------------------------------------------------------
def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (float64): biased moment estimates
    m <- beta1 m + (1 - beta1) g, v <- beta2 v + (1 - beta2) g^2, their
    bias corrections m / (1 - beta1^t), v / (1 - beta2^t), and
    theta <- theta - lr m_hat / (sqrt(v_hat) + eps).  Returns (theta, m, v)."""
    theta, g, m, v = (np.asarray(a, np.float64) for a in (theta, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


# ---------------------------------------------------------------------------
# Seeding transform (float64)
# ---------------------------------------------------------------------------
T_MIN, T_MAX = 2.7, 3000.0
FEATURE_CLIP = 6.0


def seed_features(T, rho, norm, T_prev=None, T_prev2=None):
    """Network input per cell: ((ln T - lt_mean) / lt_std, (ln rho -
    lr_mean) / lr_std); given T_prev, ((ln T - ln T_prev) - ld_mean) /
    ld_std (the last iteration's change); given T_prev2 as well, ((ln T_prev
    - ln T_prev2) - pd_mean) / pd_std (the change one iteration earlier);
    temperatures clamped to [T_MIN, T_MAX] and rho to at least 1e-30.  norm:
    dict with lt_mean, lt_std, lr_mean, lr_std (ld_mean, ld_std; pd_mean,
    pd_std).  Each standardised feature is clipped to [-FEATURE_CLIP,
    FEATURE_CLIP].  Returns (n, 2), (n, 3) or (n, 4)."""
    lT = np.log(np.clip(np.asarray(T, np.float64), T_MIN, T_MAX))
    cols = [(lT - norm["lt_mean"]) / norm["lt_std"],
            (np.log(np.maximum(np.asarray(rho, np.float64), 1e-30)) - norm["lr_mean"]) / norm["lr_std"]]
    if T_prev is not None:
        lP = np.log(np.clip(np.asarray(T_prev, np.float64), T_MIN, T_MAX))
        cols.append((lT - lP - norm["ld_mean"]) / norm["ld_std"])
        if T_prev2 is not None:
            lPP = np.log(np.clip(np.asarray(T_prev2, np.float64), T_MIN, T_MAX))
            cols.append((lP - lPP - norm["pd_mean"]) / norm["pd_std"])
    return np.clip(np.stack(cols, axis=-1), -FEATURE_CLIP, FEATURE_CLIP)


def seed_transform(T1, pred, y_mean, y_std, shrink=1.0, envelope=None):
    """T_seed = T1 exp(y), clamped to [T_MIN, T_MAX], with y = shrink (pred
    y_std + y_mean) (the network predicts the normalised ln T - ln T1) and,
    given an envelope (lnT1_lo, lnT1_hi, y_lo[n], y_hi[n]), y bounded to
    [y_lo[b], y_hi[b]] of the bin b of ln T1 (clamped to [T_MIN, T_MAX]) among
    n equal bins over [lnT1_lo, lnT1_hi), the end bins extended."""
    T1 = np.asarray(T1, np.float64)
    y = shrink * (np.asarray(pred, np.float64) * y_std + y_mean)
    if envelope is not None:
        lo, hi, ylo, yhi = envelope
        n = len(ylo)
        lt = np.log(np.clip(T1, T_MIN, T_MAX))
        b = np.clip(np.floor((lt - lo) / (hi - lo) * n).astype(np.int64), 0, n - 1)
        y = np.minimum(np.maximum(y, np.asarray(ylo, np.float64)[b]), np.asarray(yhi, np.float64)[b])
    return np.clip(T1 * np.exp(y), T_MIN, T_MAX)


def init_params(seed=0, scale=1.0):
    """He-style initial weights (the same recipe is used by the CUDA path)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, cin, cout in LAYERS:
        std = scale * np.sqrt(2.0 / (27 * cin))
        w = rng.normal(0.0, std, size=(cout, 27, cin))
        b = np.zeros(cout)
        if name == "head":
            w[1:] = 0.0
        P[name] = (w, b)
    return P
