"""The learned seed's network kernels against the FP64 oracle (oracle/nn.py),
fed the same BF16-rounded inputs and weights.  Tolerances (relative L2):
single convolutions with FP32 output 1e-4 (FP32 accumulation only); the whole
U-Net 3e-2 for the prediction and 1e-1 for the weight gradients (every layer
rounds its activations and gradients to BF16, and the first layer's gradient
sits at the end of the longest chain of such roundings)."""
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


@pytest.mark.parametrize("shape,cin,cout", [((2, 5, 6, 7), 32, 48), ((1, 9, 4, 3), 16, 16), ((1, 8, 8, 8), 192, 64),
                                             ((1, 6, 5, 4), 48, 32), ((2, 4, 4, 4), 96, 16), ((1, 4, 5, 6), 80, 256),
                                             ((1, 3, 3, 3), 320, 32)])
def test_conv3d_forward_dgrad_wgrad(libsoc, shape, cin, cout):
    rng = np.random.default_rng(cin + cout)
    x, x64 = _bf(rng.standard_normal(shape + (cin,)))
    w, w64 = _bf(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).cuda()
    y = torch.zeros(shape + (cout,), dtype=torch.float32, device="cuda")
    libsoc.conv3d(x, w, b, relu=False, out_f32=y)
    ref = O.conv3d(x64, w64, b.cpu().numpy().astype(np.float64))
    assert _rel(y.cpu().numpy(), ref) < 1e-4
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


def test_unet_forward_and_gradients_match_oracle(libsoc):
    B, S = 2, 16
    rng = np.random.default_rng(7)
    P = O.init_params(seed=1)
    for n, _, cout in O.LAYERS:
        P[n] = (P[n][0], rng.normal(0, 0.05, cout) * (np.arange(cout) < (1 if n == "head" else cout)))
    flat = _flat(P).astype(np.float32)
    net = libsoc.UNet(B, S)
    assert net.n_params == flat.size
    net.set_params(flat)
    x_np = rng.standard_normal((B, S, S, S, 2)).astype(np.float32)
    t_np = rng.standard_normal((B, S, S, S)).astype(np.float32)
    x = torch.from_numpy(x_np).cuda()
    t = torch.from_numpy(t_np).cuda()
    pred = torch.zeros((B, S, S, S), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.backward(x, t, pred, loss)
    torch.cuda.synchronize()
    # oracle on the BF16-rounded weights and inputs the network used
    Pb = {}
    for n, _, _ in O.LAYERS:
        wb = torch.from_numpy(P[n][0].astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
        Pb[n] = (wb, P[n][1].astype(np.float32).astype(np.float64))
    x16 = np.zeros((B, S, S, S, 16))
    x16[..., :2] = torch.from_numpy(x_np).to(torch.bfloat16).float().numpy()
    p_ref, cache = O.unet_forward(x16, Pb)
    assert _rel(pred.cpu().numpy(), p_ref) < 3e-2
    L_ref, g_ref = O.mse(p_ref, t_np)
    assert abs(loss.item() / L_ref - 1) < 3e-2
    G = O.unet_backward(g_ref, cache, Pb)
    g_gpu = _unflat(net.get_params(grads=True))
    for n, _, _ in O.LAYERS:
        rw = G[n][0] if n != "head" else G[n][0][:1]
        gw = g_gpu[n][0] if n != "head" else g_gpu[n][0][:1]
        assert _rel(gw, rw) < 1e-1, n
    net.close()


def test_unet_training_reduces_loss(libsoc):
    B, S = 2, 16
    rng = np.random.default_rng(3)
    net = libsoc.UNet(B, S)
    net.set_params(_flat(O.init_params(seed=2)).astype(np.float32))
    x = torch.from_numpy(rng.standard_normal((B, S, S, S, 2)).astype(np.float32)).cuda()
    # a smooth target the network can fit: a function of the inputs
    t = (0.5 * x[..., 0] - 0.3 * x[..., 1]).contiguous()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    # the weight gradient sums its split-K partials with FP32 atomics, so the
    # trajectory varies a little from run to run: 100 steps and a bound with
    # margin (the loss falls to about 0.2x of its start by step 60)
    for it in range(100):
        net.backward(x, t, loss=loss)
        net.adam(2e-3)
        hist.append(loss.item())
    assert hist[-1] < 0.25 * hist[0], hist[::10]
    assert np.mean(hist[-10:]) < 0.5 * np.mean(hist[:10]), hist[::10]
    net.close()
