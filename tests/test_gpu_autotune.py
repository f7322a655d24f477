"""Autotuner on the GPU: every candidate launch configuration must give the
same counters (the tuner raises otherwise); the winner is applied."""
import pytest

from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tuner_candidates_agree_bit_for_bit(tmp_path):
    from paper_1812_06632_gb300 import autotune as A
    w = I.config_c2(n=24, n_freq=64, n_packages=0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    specs = [dict(source=0, freq=f, n_packages=4000, tally_offset=k * cl.n_cells)
             for k, f in enumerate((5, 30, 55))]
    space = dict(threads_per_block=(64, 256), blocks_per_sm=(0, 4), chunk=(1, 16), refill=(1, 8), scatter=(1, 8))
    best, res = A.tune(ctx, specs, 3 * cl.n_cells, w.clouds, space=space, reps=1,
                       cache_path=str(tmp_path / "t.json"))
    assert len(res) == 32 and best in [c for c, _ in res]
    best2, res2 = A.tune(ctx, specs, 3 * cl.n_cells, w.clouds, space=space, cache_path=str(tmp_path / "t.json"))
    assert best2 == best


def test_tuner_candidates_agree_on_an_octree(tmp_path):
    """Octree launches keep each lane's ancestors in dynamic shared memory
    sized by the block: every block size and register build gives the same
    counters."""
    from paper_1812_06632_gb300 import autotune as A
    w = I.config_c3(root_n=8, max_refine=3, threshold=3.0, n_freq=8, tau_peak_1um=60.0)
    cl = w.clouds[0]
    assert cl.n_levels == 4
    ctx, ids = gpu_context(w)
    specs = [dict(source=s, freq=f, n_packages=3000, tally_offset=k * cl.n_cells)
             for k, (s, f) in enumerate(((0, 4), (1, 5), (1, 3)))]
    space = dict(threads_per_block=(32, 96, 256), blocks_per_sm=(0, 4), chunk=(1, 16), refill=(8,), scatter=(8,))
    best, res = A.tune(ctx, specs, 3 * cl.n_cells, w.clouds, space=space, reps=1,
                       cache_path=str(tmp_path / "o.json"))
    assert len(res) == 12 and best in [c for c, _ in res]
