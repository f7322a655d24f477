"""Surface-brightness maps (soc_map) against the FP64 exact-segment oracle:
FP32 cell-local traversal with FP64 accumulation agrees within 1e-4
relative (path lengths carry FP32 rounding)."""
import numpy as np
import pytest

import oracle
from oracle import mapping as M
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, oracle_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare(w, T, f, direction, up, npx, npy, pix, center, I_bg=0.0):
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    out = torch.zeros((npy, npx), dtype=torch.float32, device="cuda")
    ctx.map(ids[0], torch.from_numpy(T.astype(np.float32)).cuda(), f, direction, up, npx, npy, pix, center, out,
            I_bg=I_bg)
    torch.cuda.synchronize()
    g = out.cpu().numpy().astype(np.float64)
    ref = M.ray_map(oracle_grid(cl), T.astype(np.float32).astype(np.float64), w.dust.kabs[f] * cl.ell,
                    w.dust.ksca[f] * cl.ell, w.dust.nu[f], direction, up, npx, npy, pix, center, I_bg=I_bg)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(g, ref, rtol=1e-4, atol=1e-6 * scale)
    return g, ref


def test_map_lognormal_oblique():
    w = I.config_c2(n=24, n_freq=64, n_packages=0)
    cl = w.clouds[0]
    T = 10.0 + 30.0 * (cl.rho / cl.rho.max())
    g, ref = _compare(w, T, 8, [0.31, -0.42, 0.85], [0, 0, 1], 40, 36, 0.75, [12.0, 12.0, 12.0], I_bg=0.0)
    assert (g > 0).sum() > 0.5 * g.size


@pytest.mark.parametrize("direction", [[0, 0, 1], [-1, 0, 0], [0.6, 0.7, -0.3]])
def test_map_octree(direction):
    w = I.config_c3(root_n=8, max_refine=3, threshold=3.0, tau_peak_1um=50.0, n_freq=16)
    cl = w.clouds[0]
    rng = np.random.default_rng(1)
    T = rng.uniform(8.0, 200.0, cl.n_cells)
    up = [0, 1, 0] if abs(direction[1]) < 0.9 else [1, 0, 0]
    _compare(w, T, 9, direction, up, 33, 29, 0.31, [4.0, 4.0, 4.0], I_bg=1e-16)


@pytest.mark.parametrize("f,I_bg", [(36, 3e-7), (40, 3e-7), (44, 1e-6), (55, 1e-6)])
def test_map_optically_thick_with_bright_background(f, I_bg):
    """Hot dust (300-1000 K) on lines of sight of optical depth ~4, ~12, ~40
    and ~1000 across the cloud, in front of a background brighter than the
    cloud's own emission: the FP32 segment factors keep the FP64
    accumulation within the same bound."""
    w = I.config_c2(n=32, n_freq=64, n_packages=0, tau_1um=50.0)
    cl = w.clouds[0]
    T = np.random.default_rng(f).uniform(300.0, 1000.0, cl.n_cells)
    _compare(w, T, f, [0.45, 0.52, -0.73], [0, 0, 1], 48, 40, 1.1, [16.0, 16.0, 16.0], I_bg=I_bg)
