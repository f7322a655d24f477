"""The whole bench pass against the oracle: the 128^3 lognormal cloud, 64
frequencies x 1e6 background packages (7.3e9 photon-cell steps).  Every one
of the 64 x 2,097,152 int64 counters and every item's statistics must equal
the FP32-contract oracle's, which traces the same 6.4e7 packages on all host
cores (spawned processes, one frequency per task; about a minute on 16
cores)."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 1_000_000


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_W = None


def _oracle_frequency(f):
    """Counters and statistics of all N packages of frequency f (worker)."""
    global _W
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_1812_06632_gb300 import inputs as I
    from parity_helpers import oracle_item
    if _W is None:
        _W = I.config_c2()
    t, st, _ = oracle_item(_W, 0, dict(source=0, freq=f, n_packages=N))
    return f, t, st


def test_full_128cube_64nu_pass_every_counter_equals_the_oracle(libsoc):
    import oracle
    from paper_1812_06632_gb300 import inputs as I
    from parity_helpers import gpu_context, run_gpu
    oracle.build()
    w = I.config_c2()
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    specs = [dict(source=0, freq=f, n_packages=N, tally_offset=f * cl.n_cells) for f in range(nf)]
    items = ctx.items(specs)
    tally = torch.zeros(nf * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((nf, 4), dtype=torch.int64, device="cuda")
    ctx.simulate(items, tally, stats)
    torch.cuda.synchronize()
    st = stats.cpu().numpy()
    cores = max(1, min(os.cpu_count() or 1, nf))
    seen = 0
    with mp.get_context("spawn").Pool(cores) as pool:
        for f, t_o, st_o in pool.imap_unordered(_oracle_frequency, range(nf)):
            t_g = tally[f * cl.n_cells:(f + 1) * cl.n_cells].cpu().numpy()
            assert np.array_equal(t_g, t_o), f"frequency {f}: {int((t_g != t_o).sum())} counters differ"
            assert (st[f, 0], st[f, 1], st[f, 2], st[f, 3]) == \
                (st_o["escaped"], st_o["capped"], st_o["steps"], st_o["emitted"]), f
            seen += 1
    assert seen == nf
    assert int(st[:, 2].sum()) > 7e9
