"""Prepared batches and CUDA-graph replay: the captured pass (counter reset,
persistent tracer, absorbed power, temperature) gives the same counters and
temperatures as the direct calls, replay after replay; an uneven batch of
several clouds and sources runs in one launch."""
import numpy as np
import pytest

from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, oracle_item, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_graph_replay_equals_direct_calls():
    w = I.config_c2(n=32, n_freq=64, n_packages=0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    nf, N = 64, 3000
    specs = [dict(source=0, freq=f, n_packages=N, tally_offset=f * cl.n_cells) for f in range(nf)]
    ref_t, ref_s, _ = run_gpu(ctx, specs, nf * cl.n_cells, want_steps=False)
    e = torch.from_numpy(ctx.package_energy(ids[0], 0, N)).cuda()
    A_ref = torch.zeros(cl.n_cells, dtype=torch.float64, device="cuda")
    T_ref = torch.full((cl.n_cells,), 2.7, dtype=torch.float32, device="cuda")
    ctx.absorbed_power(ids[0], torch.from_numpy(ref_t).cuda(), cl.n_cells, e, A_ref)
    ctx.update_temperature(ids[0], A_ref, T_ref)
    torch.cuda.synchronize()

    bid = ctx.batch_create(ctx.items(specs))
    tally = torch.full((nf * cl.n_cells,), 7, dtype=torch.int64, device="cuda")   # garbage: must be zeroed
    stats = torch.full((nf, 4), 7, dtype=torch.int64, device="cuda")
    A = torch.zeros(cl.n_cells, dtype=torch.float64, device="cuda")
    T = torch.full((cl.n_cells,), 2.7, dtype=torch.float32, device="cuda")
    dT = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    ctx.capture_begin(s)
    ctx.batch_launch(bid, tally, stats, stream=s)
    ctx.absorbed_power(ids[0], tally, cl.n_cells, e, A, stream=s)
    ctx.update_temperature(ids[0], A, T, dT, stream=s)
    gid = ctx.capture_end(s)
    for rep in range(3):
        ctx.graph_launch(gid, stream=s)
        s.synchronize()
        np.testing.assert_array_equal(tally.cpu().numpy(), ref_t)
        np.testing.assert_array_equal(stats.cpu().numpy(), ref_s)
        np.testing.assert_array_equal(T.cpu().numpy(), T_ref.cpu().numpy())
        assert (dT.item() > 0) == (rep == 0)            # later replays: same T, max |dT| = 0
    ctx.graph_destroy(gid)
    ctx.batch_destroy(bid)


def test_uneven_cloud_batch_in_one_graph_launch():
    w = I.config_c5(n_clouds=5, n_freq=8, sizes=[16, 24, 32, 20, 28], base_packages=1500)
    ctx, ids = gpu_context(w)
    specs, offs, off = [], [], 0
    for ci, cl in enumerate(w.clouds):
        for src in (0, 1):
            for f in range(0, 8, 3):
                specs.append(dict(cloud=ids[ci], source=src, freq=f, n_packages=w.n_bg[ci] // 4, tally_offset=off))
                offs.append((ci, off))
                off += cl.n_cells
    ref = run_gpu(ctx, specs, off, want_steps=False)
    bid = ctx.batch_create(ctx.items(specs))
    tally = torch.zeros(off, dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    ctx.capture_begin(s)
    ctx.batch_launch(bid, tally, stats, stream=s)
    gid = ctx.capture_end(s)
    ctx.graph_launch(gid, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(tally.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(stats.cpu().numpy(), ref[1])
    # two items against the oracle directly
    t = tally.cpu().numpy()
    for k in (1, len(specs) - 1):
        ci, o = offs[k]
        t_o = oracle_item(w, ci, specs[k])[0]
        np.testing.assert_array_equal(t[o:o + w.clouds[ci].n_cells], t_o)
