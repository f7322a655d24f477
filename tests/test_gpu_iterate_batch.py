"""soc_iterate_batch: several clouds iterated together, one tracer launch per
iteration for all clouds not yet converged.  Each cloud's temperatures,
iteration count and photon-cell steps must equal those of soc_iterate on
that cloud alone, bit for bit (the packages, their random numbers and their
integer counters do not depend on which launch carries them), with and
without seeds, with the diagonal operator, and across a reused iteration 0.
The per-cloud runs are themselves matched against the oracle-driven
iteration in tests/test_gpu_parity.py."""
import numpy as np
import pytest

from paper_1812_06632_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _clouds():
    """Three clouds of uneven size (two regular grids and an octree) on one
    shared dust table, each with a point source and the background."""
    wo = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0, tau_peak_1um=60.0, n_freq=16,
                     n_bg=20_000, n_ps=20_000, L_bol=3e36, side_pc=0.05)
    ell = wo.clouds[0].ell
    regs = [I.regular(I.lognormal_density(n, s, 1.5, -3.5).astype(np.float32) * np.float32(f), ell=ell)
            for n, s, f in ((16, 4, 30.0), (24, 5, 8.0))]
    nu = wo.dust.nu
    L = wo.ps_L[0][:1]
    return I.Workload("batch3", [regs[0], wo.clouds[0], regs[1]], wo.dust, [I.diluted_blackbodies(nu)] * 3,
                      [np.array([[8.0, 8.5, 7.5]]), wo.ps_pos[0][:1], np.array([[12.0, 11.0, 12.5]])],
                      [L, L, L], [20_000] * 3, [20_000] * 3, seed=5)


def _ctx(w, soc):
    ctx = soc.Context(0, w.seed)
    ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    ids = []
    for ci, cl in enumerate(w.clouds):
        cid = ctx.grid_upload(cl)
        ctx.sources_upload(cid, w.bg_I[ci], w.ps_pos[ci], w.ps_L[ci])
        ids.append(cid)
    return ctx, ids


@pytest.mark.parametrize("ali", [False, True])
def test_batch_equals_per_cloud_iterations(libsoc, ali):
    w = _clouds()
    kw = dict(n_background=20_000, n_point=20_000, n_per_cell=1, max_iter=40, dT_tol=0.1, ali=ali)
    ref_ctx, ids = _ctx(w, libsoc)
    ref = []
    for k, cid in enumerate(ids):
        T = torch.zeros(w.clouds[k].n_cells, dtype=torch.float32, device="cuda")
        r = ref_ctx.iterate(cid, T, **kw)
        ref.append((T.cpu().numpy(), r))
    ctx, ids2 = _ctx(w, libsoc)
    assert ids2 == ids
    Ts = [torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda") for cl in w.clouds]
    rows, timed_out = ctx.iterate_batch(ids2, Ts, **kw)
    assert not timed_out
    for k in range(3):
        np.testing.assert_array_equal(Ts[k].cpu().numpy(), ref[k][0])
        assert rows[k]["iterations"] == ref[k][1]["iterations"]
        assert rows[k]["converged"] == ref[k][1]["converged"]
        assert rows[k]["steps"] == ref[k][1]["steps"]
        np.testing.assert_array_equal(rows[k]["history"], ref[k][1]["history"])
    assert any(r["converged"] for r in rows)
    # clouds leave the batch at different iterations
    assert len({r["iterations"] for r in rows}) > 1 or not all(r["converged"] for r in rows)


def test_batch_with_seeds_and_reused_iteration0(libsoc):
    w = _clouds()
    ref_ctx, ids = _ctx(w, libsoc)
    ctx, ids2 = _ctx(w, libsoc)
    n = [cl.n_cells for cl in w.clouds]
    # iteration 0 only, batched and per cloud
    T1 = [torch.zeros(m, dtype=torch.float32, device="cuda") for m in n]
    rows0, _ = ctx.iterate_batch(ids2, T1, n_background=20_000, n_point=20_000, max_iter=0)
    assert all(r["iterations"] == 0 for r in rows0)
    T1_ref = []
    for k, cid in enumerate(ids):
        T = torch.zeros(n[k], dtype=torch.float32, device="cuda")
        ref_ctx.iterate(cid, T, n_background=20_000, n_point=20_000, max_iter=0)
        T1_ref.append(T)
        np.testing.assert_array_equal(T1[k].cpu().numpy(), T.cpu().numpy())
    # seeds for clouds 0 and 2 (T1 scaled up), cloud 1 from the constant sources
    seeds = [(T1[0] * 1.3).contiguous(), None, (T1[2] * 0.8).contiguous()]
    Ts = [torch.zeros(m, dtype=torch.float32, device="cuda") for m in n]
    rows, _ = ctx.iterate_batch(ids2, Ts, n_per_cell=1, max_iter=30, dT_tol=0.1, T_seeds=seeds, reuse_constant=True)
    for k, cid in enumerate(ids):
        T = torch.zeros(n[k], dtype=torch.float32, device="cuda")
        r = ref_ctx.iterate(cid, T, n_per_cell=1, max_iter=30, dT_tol=0.1, T_seed=seeds[k], reuse_constant=True)
        np.testing.assert_array_equal(Ts[k].cpu().numpy(), T.cpu().numpy())
        assert rows[k]["iterations"] == r["iterations"] and rows[k]["steps"] == r["steps"]


def test_batch_argument_checks(libsoc):
    w = _clouds()
    ctx, ids = _ctx(w, libsoc)
    Ts = [torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda") for cl in w.clouds]
    with pytest.raises(libsoc.SocError):                      # a cloud twice
        ctx.iterate_batch([ids[0], ids[0]], Ts[:1] * 2, max_iter=1)
    with pytest.raises(libsoc.SocError):                      # iteration 0 was never run
        ctx.iterate_batch(ids, Ts, max_iter=1, reuse_constant=True)


def test_sharded_driver_on_the_library_equals_soc_iterate(libsoc):
    """shard.iterate_sharded with the library as its backend (one rank: the
    counter all-reduce is the identity) reproduces soc_iterate bit for bit;
    the same driver on two gloo ranks reproduces one rank (test_shard_gloo)."""
    from paper_1812_06632_gb300 import shard
    w = _clouds()
    kw = dict(n_background=20_000, n_point=20_000, n_per_cell=1, max_iter=6, dT_tol=0.1)
    ref_ctx, ids = _ctx(w, libsoc)
    ctx, ids2 = _ctx(w, libsoc)
    for k in (0, 1):
        cl = w.clouds[k]
        T_ref = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
        r_ref = ref_ctx.iterate(ids[k], T_ref, **kw)
        be = shard.LibraryBackend(ctx, ids2[k], cl.n_cells, cl.leaves().size, len(w.dust.nu))
        T = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
        r = shard.iterate_sharded(be, T, **kw)
        np.testing.assert_array_equal(T.cpu().numpy(), T_ref.cpu().numpy())
        assert r["iterations"] == r_ref["iterations"] and r["steps"] == r_ref["steps"]
        np.testing.assert_array_equal(np.array(r["history"]), r_ref["history"])
