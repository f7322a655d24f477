"""The abort flag and the soc_iterate watchdog (SOC_ERR_TIMEOUT).

The failure is made on the host: the test sets the context's abort flag
(soc_abort) or lets the watchdog deadline of soc_set_timeout pass.  No GPU
fault, trap or hang is involved: tracer warps read the flag when they take a
new chunk of work and simply stop taking work, so every wait stays bounded.
What was traced before the stop must still conserve energy exactly.
"""
import time

import numpy as np
import pytest

from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _per_item_conservation(tally, stats, n_items, n_cells):
    """sum(tally of item) + escaped == emitted, exactly, for every item."""
    dep = tally.view(n_items, n_cells).sum(1)
    torch.testing.assert_close(dep + stats[:, 0], stats[:, 3], rtol=0, atol=0)


def test_abort_before_launch_traces_nothing_and_clear_restores():
    w = I.config_c2(n=32, n_freq=8, n_packages=0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    specs = [dict(source=0, freq=f, n_packages=4000, tally_offset=f * cl.n_cells) for f in range(8)]
    ref = run_gpu(ctx, specs, 8 * cl.n_cells)
    assert ctx.abort_status() == (False, False)
    ctx.abort()
    t, st, steps = run_gpu(ctx, specs, 8 * cl.n_cells)
    assert not t.any() and not st.any() and not steps.any()
    assert ctx.abort_status() == (True, True)
    ctx.abort_clear()
    assert ctx.abort_status() == (False, False)
    got = run_gpu(ctx, specs, 8 * cl.n_cells)
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_abort_during_a_long_launch_conserves_what_was_traced():
    w = I.config_c2(n=128, n_freq=64, n_packages=0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    nf, N = 64, 1_000_000
    specs = [dict(source=0, freq=f, n_packages=N, tally_offset=f * cl.n_cells) for f in range(nf)]
    items = ctx.items(specs)
    tally = torch.zeros(nf * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((nf, 4), dtype=torch.int64, device="cuda")
    # warm-up launch of a few packages (module load, first-touch of the grid)
    ctx.simulate(ctx.items(specs[:1]), tally, stats[:1])
    torch.cuda.synchronize()
    tally.zero_(); stats.zero_()
    torch.cuda.synchronize()
    ctx.simulate(items, tally, stats)        # ~65 ms on GB300
    time.sleep(0.01)
    ctx.abort()
    torch.cuda.synchronize()
    requested, cut = ctx.abort_status()
    assert requested and cut
    emitted = int(stats[:, 3].sum())
    assert 0 < emitted < nf * N * (1 << 31)
    _per_item_conservation(tally, stats, nf, cl.n_cells)
    ctx.abort_clear()


def test_graph_replay_reads_the_flag():
    w = I.config_c2(n=32, n_freq=4, n_packages=0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    specs = [dict(source=0, freq=f, n_packages=3000, tally_offset=f * cl.n_cells) for f in range(4)]
    ref = run_gpu(ctx, specs, 4 * cl.n_cells, want_steps=False)
    bid = ctx.batch_create(ctx.items(specs))
    tally = torch.zeros(4 * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((4, 4), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    ctx.capture_begin(s)
    ctx.batch_launch(bid, tally, stats, stream=s)
    gid = ctx.capture_end(s)
    ctx.abort()
    ctx.graph_launch(gid, stream=s)
    s.synchronize()
    assert not tally.any().item() and not stats.any().item()
    ctx.abort_clear()
    ctx.graph_launch(gid, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(tally.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(stats.cpu().numpy(), ref[1])
    ctx.graph_destroy(gid)
    ctx.batch_destroy(bid)


def test_iterate_watchdog_returns_timeout_with_partial_result():
    w = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0, tau_peak_1um=30.0, n_freq=16,
                    n_bg=20_000, n_ps=20_000)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    T = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
    # a deadline far shorter than 500 dust iterations with an unreachable tolerance
    ctx.set_timeout(0.05)
    t0 = time.perf_counter()
    r = ctx.iterate(ids[0], T, n_background=20_000, n_point=20_000, max_iter=500, dT_tol=0.0)
    wall = time.perf_counter() - t0
    assert r["timed_out"] and not r["converged"]
    assert r["iterations"] < 500 and wall < 5.0
    assert ctx.abort_status()[0]
    assert np.isfinite(T.cpu().numpy()).all()
    # the flag is sticky: the next call stops at once
    r2 = ctx.iterate(ids[0], T, n_background=20_000, n_point=20_000, max_iter=3, dT_tol=0.0)
    assert r2["timed_out"] and r2["iterations"] == 0
    ctx.abort_clear()
    ctx.set_timeout(0.0)
    r3 = ctx.iterate(ids[0], T, n_background=20_000, n_point=20_000, max_iter=3, dT_tol=0.0)
    assert not r3["timed_out"] and r3["iterations"] == 3
