"""The learned seed's network kernels against the FP64 oracle (oracle/nn.py),
fed the same BF16-rounded inputs and weights.  Tolerances (relative L2):
single convolutions with FP32 output 1e-4 (FP32 accumulation only).  The
whole U-Net is compared with the oracle run at the network's stated
precision (every stored activation and every layer's output gradient rounded
to BF16 at the points where the kernels store them, arithmetic in FP64): the
two then differ only by FP32 accumulation order and the rare BF16 rounding it
flips, so the prediction and every layer's weight and bias gradient are held
to per-layer bounds far below the size of BF16 rounding itself (which moves
the first layer's weight gradient by ~10 %).  Adam and the seeding transform
are compared element by element; training is bit-reproducible."""
import numpy as np
import pytest

from oracle import nn as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf(a):
    """BF16 device tensor and its exact FP64 value."""
    h = torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16)      # rounded on the host
    return h.cuda(), h.float().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# The first seven shapes take the per-tap kernel; the others the slab-fed
# one: rows of 64, 32 and 16 voxels; y and z tails shorter than the output
# box; 1 to 3 K chunks of 16 or 32 channels; up to 16 channel tiles; 1, 2
# or 4 accumulator groups; channel tiles of 16, 32 and 48 (the last with all
# 512 tensor-memory columns, three stages and one block per SM), in the
# forward direction and, for several, in the input gradient as well (the
# plans the U-Net's 64^3 training takes).
@pytest.mark.parametrize("shape,cin,cout", [((2, 5, 6, 7), 32, 48), ((1, 9, 4, 3), 16, 16), ((1, 8, 8, 8), 192, 64),
                                             ((1, 6, 5, 4), 48, 32), ((2, 4, 4, 4), 96, 16), ((1, 4, 5, 6), 80, 256),
                                             ((1, 3, 3, 3), 320, 32), ((1, 9, 7, 64), 16, 256),
                                             ((2, 13, 10, 32), 48, 160), ((4, 16, 16, 16), 64, 64),
                                             ((4, 32, 32, 32), 16, 32), ((4, 16, 16, 16), 64, 32),
                                             ((1, 76, 16, 64), 16, 48), ((3, 32, 16, 32), 32, 96)])
def test_conv3d_forward_dgrad_wgrad(libsoc, shape, cin, cout):
    rng = np.random.default_rng(cin + cout)
    x, x64 = _bf(rng.standard_normal(shape + (cin,)))
    w, w64 = _bf(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).cuda()
    y = torch.zeros(shape + (cout,), dtype=torch.float32, device="cuda")
    libsoc.conv3d(x, w, b, relu=False, out_f32=y)
    ref = O.conv3d(x64, w64, b.cpu().numpy().astype(np.float64))
    assert _rel(y.cpu().numpy(), ref) < 1e-4
    # every output (a voxel or channel mapped to the wrong accumulator row or
    # column is off by the order of the outputs themselves)
    assert np.abs(y.cpu().numpy() - ref).max() < 1e-3 * max(np.abs(ref).max(), 1.0)
    # BF16 output with ReLU
    y16 = torch.zeros(shape + (cout,), dtype=torch.bfloat16, device="cuda")
    libsoc.conv3d(x, w, b, relu=True, out=y16)
    assert _rel(y16.float().cpu().numpy(), np.maximum(ref, 0)) < 1e-2
    # gradients
    gy, gy64 = _bf(rng.standard_normal(shape + (cout,)))
    gx = torch.zeros(shape + (cin,), dtype=torch.float32, device="cuda")
    scratch = torch.empty(cout * 27 * cin, dtype=torch.bfloat16, device="cuda")
    libsoc.conv3d_dgrad(gy, w, scratch, gx)
    assert _rel(gx.cpu().numpy(), O.conv3d_dgrad(gy64, w64)) < 1e-4
    gw = torch.zeros((cout, 27, cin), dtype=torch.float32, device="cuda")
    gb = torch.zeros(cout, dtype=torch.float32, device="cuda")
    libsoc.conv3d_wgrad(gy, x, gw, gb)
    rw, rb = O.conv3d_wgrad(gy64, x64)
    assert _rel(gw.cpu().numpy(), rw) < 1e-4
    assert _rel(gb.cpu().numpy(), rb) < 1e-4


def _flat(P):
    return np.concatenate([np.concatenate([P[n][0].ravel(), P[n][1].ravel()]) for n, _, _ in O.LAYERS])


def _unflat(flat):
    P, k = {}, 0
    for n, cin, cout in O.LAYERS:
        nw = cout * 27 * cin
        P[n] = (flat[k:k + nw].reshape(cout, 27, cin).astype(np.float64), flat[k + nw:k + nw + cout].astype(np.float64))
        k += nw + cout
    return P


def _bf_params(P):
    """The weights the network uses: BF16-rounded weights, FP32 biases."""
    Pb = {}
    for n, _, _ in O.LAYERS:
        wb = torch.from_numpy(P[n][0].astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
        Pb[n] = (wb, P[n][1].astype(np.float32).astype(np.float64))
    return Pb


# Per-layer relative L2 bounds of the weight and bias gradients, and of the
# prediction, against the BF16-storage oracle.  Measured on GB300 (seeds 7
# and 8): at 32^3 the weight gradients differ by 0.01-2.8 % (largest at the
# first layer and the 8^3-4^3 bottleneck layers), the biases by up to 1.8 %,
# the prediction by 0.5-0.6 %; at 16^3 by up to 7.3 % -- the differences
# shrink as the layers' reductions run over more voxels, as independent
# rounding differences (FP32 tensor-core accumulation flipping BF16 roundings
# of stored activations and gradients) do, while a wrong term or index would
# not shrink.  Bounds: about twice the largest measured value.
GRAD_BOUND_W, GRAD_BOUND_B, PRED_BOUND = 6e-2, 4e-2, 1.5e-2


@pytest.mark.parametrize("n_in", [2, 3])
def test_unet_forward_and_gradients_match_oracle(libsoc, n_in):
    B, S = 1, 32
    rng = np.random.default_rng(7)
    P = O.init_params(seed=1)
    for n, _, cout in O.LAYERS:
        P[n] = (P[n][0], rng.normal(0, 0.05, cout) * (np.arange(cout) < (1 if n == "head" else cout)))
    flat = _flat(P).astype(np.float32)
    net = libsoc.UNet(B, S, n_inputs=n_in)
    assert net.n_params == flat.size
    net.set_params(flat)
    x_np = rng.standard_normal((B, S, S, S, n_in)).astype(np.float32)
    t_np = rng.standard_normal((B, S, S, S)).astype(np.float32)
    x = torch.from_numpy(x_np).cuda()
    t = torch.from_numpy(t_np).cuda()
    pred = torch.zeros((B, S, S, S), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.backward(x, t, pred, loss)
    torch.cuda.synchronize()
    Pb = _bf_params(P)
    x16 = np.zeros((B, S, S, S, 16))
    x16[..., :n_in] = torch.from_numpy(x_np).to(torch.bfloat16).float().numpy()
    p_ref, cache = O.unet_forward(x16, Pb, store_bf16=True)
    assert _rel(pred.cpu().numpy(), p_ref) < PRED_BOUND
    L_ref, g_ref = O.mse(p_ref, t_np)
    assert abs(loss.item() / L_ref - 1) < 1e-3
    # the gradient the network back-propagates is the one of its own FP32
    # prediction (2 (pred - t) / V), so the oracle's backward starts there
    g_pred = 2.0 * (pred.cpu().numpy().astype(np.float64) - t_np) / t_np.size
    G = O.unet_backward(g_pred, cache, Pb, store_bf16=True)
    g_gpu = _unflat(net.get_params(grads=True))
    errs = {}
    for n, _, _ in O.LAYERS:
        rw = G[n][0] if n != "head" else G[n][0][:1]
        gw = g_gpu[n][0] if n != "head" else g_gpu[n][0][:1]
        rb = G[n][1] if n != "head" else G[n][1][:1]
        gb = g_gpu[n][1] if n != "head" else g_gpu[n][1][:1]
        errs[n] = (_rel(gw, rw), _rel(gb, rb))
    assert all(e[0] < GRAD_BOUND_W and e[1] < GRAD_BOUND_B for e in errs.values()), errs
    # the layers nearest the loss agree far more closely
    assert errs["head"][0] < 1e-3 and errs["d0b"][0] < 5e-3, errs
    net.close()


def _adam_ref(w, g, m, v, t, lr):
    """The oracle's Adam with the kernel's FP32 constants."""
    return O.adam_step(w, g, m, v, t, lr, beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)),
                       eps=float(np.float32(1e-8)))


def _close_to_fp32(got, ref, terms, scale):
    """|got - ref| <= 4 ulp(largest term of the FP32 sum) + 2e-6 scale,
    element-wise: a sum of FP32 terms carries the rounding of its largest
    term even where the terms cancel."""
    big = np.max(np.abs(np.stack([np.asarray(t, np.float64) * np.ones_like(ref) for t in terms])), axis=0)
    tol = 4 * np.spacing(big.astype(np.float32)).astype(np.float64) + 2e-6 * np.abs(scale)
    bad = np.abs(got.astype(np.float64) - ref) > tol
    assert not bad.any(), (int(bad.sum()), np.flatnonzero(bad)[:5])


def test_adam_kernel_matches_oracle_elementwise(libsoc):
    rng = np.random.default_rng(21)
    n = 100_003
    w = rng.standard_normal(n).astype(np.float32)
    g = (rng.standard_normal(n) * 10.0 ** rng.integers(-4, 3, n)).astype(np.float32)
    g[::97] = 0.0
    m = (rng.standard_normal(n) * 0.1).astype(np.float32)
    v = (rng.random(n) * 0.01).astype(np.float32)
    for t in (1, 2, 7, 1000):
        lr = 1e-3
        wd, md, vd, gd = (torch.from_numpy(a.copy()).cuda() for a in (w, m, v, g))
        w16 = torch.empty(n, dtype=torch.bfloat16, device="cuda")
        libsoc.adam(wd, md, vd, gd, lr, t, w16)
        torch.cuda.synchronize()
        rw, rm, rv = _adam_ref(w, g, m, v, t, lr)
        step = rw - w.astype(np.float64)
        g64 = g.astype(np.float64)
        _close_to_fp32(md.cpu().numpy(), rm, [0.9 * m, 0.1 * g64], rm)
        _close_to_fp32(vd.cpu().numpy(), rv, [0.999 * v, 0.001 * g64 * g64], rv)
        _close_to_fp32(wd.cpu().numpy(), rw, [w, step], step)
        np.testing.assert_array_equal(w16.float().cpu().numpy(), O.bf16(wd.cpu().numpy()))


def test_unet_adam_steps_match_oracle(libsoc):
    """Two soc_unet_adam steps on the network's own gradients equal the
    oracle's Adam replayed on the same gradients."""
    B, S = 1, 16
    rng = np.random.default_rng(22)
    net = libsoc.UNet(B, S)
    w0 = _flat(O.init_params(seed=4)).astype(np.float32)
    net.set_params(w0)
    x = torch.from_numpy(rng.standard_normal((B, S, S, S, 2)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, S, S, S)).astype(np.float32)).cuda()
    lr = 3e-3
    w, m, v = w0.astype(np.float64), np.zeros(w0.size), np.zeros(w0.size)
    for step in (1, 2):
        net.backward(x, t)
        g = net.get_params(grads=True)
        net.adam(lr)
        w_gpu = net.get_params()
        w_ref, m, v = _adam_ref(w.astype(np.float32), g, m, v, step, lr)
        _close_to_fp32(w_gpu, w_ref, [w, lr], lr)
        w = w_gpu.astype(np.float64)
    net.close()


def _train(libsoc, steps, seed=3):
    B, S = 2, 16
    rng = np.random.default_rng(seed)
    net = libsoc.UNet(B, S)
    net.set_params(_flat(O.init_params(seed=2)).astype(np.float32))
    x = torch.from_numpy(rng.standard_normal((B, S, S, S, 2)).astype(np.float32)).cuda()
    # a smooth target the network can fit: a function of the inputs
    t = (0.5 * x[..., 0] - 0.3 * x[..., 1]).contiguous()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    for it in range(steps):
        net.backward(x, t, loss=loss)
        net.adam(2e-3)
        hist.append(loss.item())
    w = net.get_params()
    net.close()
    return np.array(hist), w


def test_unet_training_reduces_loss_and_is_bit_reproducible(libsoc):
    """Every reduction is an ordered sum of per-block partials, so two runs
    from the same start give identical losses and weights, bit for bit."""
    h1, w1 = _train(libsoc, 80)
    h2, w2 = _train(libsoc, 80)
    np.testing.assert_array_equal(h1, h2)
    np.testing.assert_array_equal(w1, w2)
    assert h1[-1] < 0.2 * h1[0], h1[::10]


def test_seed_features_and_transform_match_oracle(libsoc):
    from parity_helpers import gpu_context
    from paper_1812_06632_gb300 import inputs as I
    w = I.config_c2(n=16, n_freq=4, n_packages=0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    rng = np.random.default_rng(23)
    T1 = rng.uniform(1.0, 400.0, cl.n_cells).astype(np.float32)
    T1[:5] = [0.5, 2.7, 3000.0, 5000.0, 20.0]
    norm = dict(lt_mean=3.1, lt_std=0.7, lr_mean=-0.2, lr_std=1.4)
    x = torch.empty((cl.n_cells, 2), dtype=torch.float32, device="cuda")
    T1d = torch.from_numpy(T1).cuda()
    ctx.seed_features(ids[0], T1d, [norm["lt_mean"], norm["lt_std"], norm["lr_mean"], norm["lr_std"]], x)
    pred = rng.standard_normal(cl.n_cells).astype(np.float32)
    pred[:3] = [40.0, -40.0, 0.0]
    Ts = torch.empty(cl.n_cells, dtype=torch.float32, device="cuda")
    ctx.seed_transform(ids[0], T1d, torch.from_numpy(pred).cuda(), libsoc.seed_map(0.15, 0.6), Ts)
    torch.cuda.synchronize()
    xr = O.seed_features(T1, cl.rho.astype(np.float32), norm)
    np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=2e-7, atol=2e-7)
    # three features: the last iteration's change of ln T as well
    Tp = (T1 * rng.uniform(0.5, 1.0, cl.n_cells)).astype(np.float32)
    norm3 = dict(norm, ld_mean=0.2, ld_std=0.3)
    x3 = torch.empty((cl.n_cells, 3), dtype=torch.float32, device="cuda")
    ctx.seed_features(ids[0], T1d, [3.1, 0.7, -0.2, 1.4, 0.2, 0.3], x3, T_prev=torch.from_numpy(Tp).cuda())
    torch.cuda.synchronize()
    np.testing.assert_allclose(x3.cpu().numpy(), O.seed_features(T1, cl.rho.astype(np.float32), norm3, T_prev=Tp),
                               rtol=2e-7, atol=2e-7)
    # four features: the change one iteration earlier too
    Tpp = (Tp * rng.uniform(0.5, 1.0, cl.n_cells)).astype(np.float32)
    norm4 = dict(norm3, pd_mean=0.25, pd_std=0.35)
    x4 = torch.empty((cl.n_cells, 4), dtype=torch.float32, device="cuda")
    ctx.seed_features(ids[0], T1d, [3.1, 0.7, -0.2, 1.4, 0.2, 0.3, 0.25, 0.35], x4, T_prev=torch.from_numpy(Tp).cuda(),
                      T_prev2=torch.from_numpy(Tpp).cuda())
    torch.cuda.synchronize()
    np.testing.assert_allclose(x4.cpu().numpy(),
                               O.seed_features(T1, cl.rho.astype(np.float32), norm4, T_prev=Tp, T_prev2=Tpp),
                               rtol=2e-7, atol=2e-7)
    with pytest.raises(libsoc.SocError):                      # four features without T_prev2
        ctx.seed_features(ids[0], T1d, [3.1, 0.7, -0.2, 1.4, 0.2, 0.3, 0.25, 0.35], x4,
                          T_prev=torch.from_numpy(Tp).cuda())
    Tr = O.seed_transform(T1, pred, 0.15, 0.6)
    np.testing.assert_allclose(Ts.cpu().numpy(), Tr, rtol=2e-7)
    # shrink and a 64-bin envelope; cells within 1e-9 of a bin edge are left
    # out (their bin can differ with the last bit of ln T1)
    n = 64
    lo, hi = float(np.log(2.7)), float(np.log(3000.0))
    ylo = np.linspace(0.0, 0.3, n)
    yhi = ylo + np.linspace(1.5, 0.1, n)
    env = (lo, hi, ylo, yhi)
    ctx.seed_transform(ids[0], T1d, torch.from_numpy(pred).cuda(), libsoc.seed_map(0.15, 0.6, 0.7, env), Ts)
    torch.cuda.synchronize()
    Tr = O.seed_transform(T1, pred, 0.15, 0.6, shrink=0.7, envelope=env)
    u = (np.log(np.clip(T1.astype(np.float64), 2.7, 3000.0)) - lo) / (hi - lo) * n
    ok = np.abs(u - np.round(u)) > 1e-9
    assert ok.sum() > 0.99 * ok.size
    np.testing.assert_allclose(Ts.cpu().numpy()[ok], Tr[ok], rtol=2e-7)
    assert (Tr != O.seed_transform(T1, pred, 0.15, 0.6, shrink=0.7)).any()      # the envelope binds somewhere
    # an octree is refused
    wo = I.config_c3(root_n=8, max_refine=1, n_freq=4, n_bg=0, n_ps=0)
    ctx2, ids2 = gpu_context(wo)
    with pytest.raises(libsoc.SocError):
        ctx2.seed_features(ids2[0], torch.zeros(wo.clouds[0].n_cells, device="cuda"), [0, 1, 0, 1],
                           torch.empty((wo.clouds[0].n_cells, 2), device="cuda"))


def test_scale_add_is_one_fused_multiply_add_per_element(libsoc):
    """soc_nn_scale_add (the ensemble's mean): y <- fma(a, x, y), a ragged
    length.  The FP64 sum of the exact product a x (48 bits) and y, rounded
    to FP32, is the fused result except when the FP64 rounding of the sum
    lands on an FP32 tie (double rounding): allow 1 ulp on at most a few
    elements."""
    rng = np.random.default_rng(11)
    n = 1_000_003
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    a = np.float32(1.0 / 3.0)
    yd = torch.from_numpy(y).cuda()
    libsoc.scale_add(yd, torch.from_numpy(x).cuda(), float(a))
    got = yd.cpu().numpy()
    ref = (np.float64(a) * x.astype(np.float64) + y.astype(np.float64)).astype(np.float32)
    ulp = np.abs(got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1 and int((ulp > 0).sum()) <= 10
    with pytest.raises(ValueError):
        libsoc.scale_add(yd, torch.zeros(3, device="cuda"), 1.0)
