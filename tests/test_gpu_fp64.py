"""The GPU's counters against the FP64 Monte Carlo oracle: the error of the
FP32 stepping stated on the device's own output (the same bounds as the
FP32-contract oracle meets against FP64)."""
import numpy as np
import pytest

import oracle
from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, kappa_root, oracle_grid, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("wl,src,f", [("c2", 0, 10), ("c2", 0, 50), ("oct", 0, 5), ("oct", 1, 5)])
def test_gpu_counters_against_fp64(wl, src, f):
    w = (I.config_c2(n_packages=0) if wl == "c2"
         else I.config_c3(root_n=16, max_refine=3, threshold=3.0, n_freq=8, tau_peak_1um=50.0))
    cl = w.clouds[0]
    n = 3000
    ctx, ids = gpu_context(w)
    t_gpu, st_gpu, n_gpu = run_gpu(ctx, [dict(source=src, freq=f, n_packages=n, tally_offset=0)], cl.n_cells)
    ka, ks = kappa_root(w.dust, f, cl.ell)
    kw = dict(source=src, kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed, freq=f, n_packages=n,
              want_steps=True)
    if src == 1:
        kw["ps_pos"] = np.asarray(w.ps_pos[0], np.float64).astype(np.float32)
        kw["ps_cdf"] = P.point_source_cdf(w.ps_L[0])[f]
    t64, s64, n64 = oracle.trace64(oracle_grid(cl), **kw)
    E = s64["emitted"]
    assert st_gpu[0][3] == E
    assert np.mean(n_gpu == n64) >= 0.97
    assert abs(float(t_gpu.sum()) - t64.sum()) <= 1e-6 * E
    assert abs(st_gpu[0][0] - s64["escaped"]) <= 1e-6 * E
    assert np.abs(t_gpu - t64).sum() <= 3e-4 * t64.sum()
