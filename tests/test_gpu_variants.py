"""Parity of the tracer builds the library picks per launch (one cloud in the
kernel parameters or each lane's own cloud; two steps per pass on regular
grids or one on octrees; with or without the ALI self counters), and of the
octree and uneven-batch workloads at full size, on sampled packages the
oracle replays one by one plus exact conservation of every item."""
import numpy as np
import pytest

import oracle
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, kappa_root, oracle_grid, oracle_item, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mixed_workload():
    """A small octree (with point sources) and a regular lognormal cube in
    one workload: a launch over both uses each lane's own cloud and one step
    per pass."""
    w = I.config_c3(root_n=6, max_refine=2, sigma=2.0, threshold=3.0, n_freq=8, tau_peak_1um=40.0)
    reg = I.config_c2(n=12, n_freq=8, n_packages=0, tau_1um=3.0)
    w.clouds.append(reg.clouds[0])
    w.bg_I.append(reg.bg_I[0])
    w.ps_pos.append(None)
    w.ps_L.append(None)
    w.n_bg.append(0)
    w.n_ps.append(0)
    return w


def _dust_weights(n, seed):
    return np.random.default_rng(seed).integers(1, 2 ** 31, n).astype(np.uint64)


@pytest.mark.parametrize("self_counters", [False, True])
def test_mixed_regular_and_octree_launch_bit_exact(self_counters):
    w = _mixed_workload()
    ctx, ids = gpu_context(w)
    dws = [_dust_weights(cl.leaves().size, 40 + ci) for ci, cl in enumerate(w.clouds)]
    dw_dev = [torch.from_numpy(d.view(np.int64)).cuda() for d in dws]
    specs, meta, off = [], [], 0
    for ci, cl in enumerate(w.clouds):
        srcs = [(0, 900), (2, cl.leaves().size)] + ([(1, 700)] if ci == 0 else [])
        for src, n in srcs:
            for f in (2, 6):
                s = dict(cloud=ids[ci], source=src, freq=f, n_packages=n, tally_offset=off, iteration=1)
                if src == 2:
                    s["dust_w"] = dw_dev[ci]
                specs.append(s)
                meta.append((ci, off))
                off += cl.n_cells
    items = ctx.items(specs)
    tally = torch.zeros(off, dtype=torch.int64, device="cuda")
    selft = torch.zeros(off, dtype=torch.int64, device="cuda") if self_counters else None
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    steps = torch.zeros(sum(s["n_packages"] for s in specs), dtype=torch.int32, device="cuda")
    ctx.simulate(items, tally, stats, steps, self_tally=selft)
    torch.cuda.synchronize()
    t, st = tally.cpu().numpy(), stats.cpu().numpy()
    sp = steps.cpu().numpy().view(np.uint32)
    sf = selft.cpu().numpy() if self_counters else None
    p = 0
    for k, s in enumerate(specs):
        ci, o = meta[k]
        cl = w.clouds[ci]
        spec = dict(s, cloud=ci)
        spec.pop("dust_w", None)
        n = s["n_packages"]
        if self_counters:
            so = np.zeros(cl.n_cells, np.int64)
            f = s["freq"]
            ka, ks = kappa_root(w.dust, f, cl.ell)
            kw = dict(source=s["source"], kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed, freq=f,
                      iteration=1, cloud=ci, n_packages=n, self_tally=so, want_steps=True)
            if s["source"] == 1:
                from oracle import physics as P
                kw["ps_pos"] = np.asarray(w.ps_pos[ci], np.float64).astype(np.float32)
                kw["ps_cdf"] = P.point_source_cdf(w.ps_L[ci])[f]
            if s["source"] == 2:
                kw.update(leaf=cl.leaves(), dust_w=dws[ci], n_per_cell=1)
            to, sto, so_steps = oracle.trace(oracle_grid(cl), **kw)
            np.testing.assert_array_equal(sf[o:o + cl.n_cells], so)
        else:
            to, sto, so_steps = oracle_item(w, ci, spec, dust_w=dws[ci] if s["source"] == 2 else None)
        np.testing.assert_array_equal(t[o:o + cl.n_cells], to)
        assert st[k][0] == sto["escaped"] and st[k][2] == sto["steps"] and st[k][3] == sto["emitted"]
        np.testing.assert_array_equal(sp[p:p + n], so_steps)
        p += n


def _sample_and_check(w, ci, specs, k_items, steps_dev, starts, rng, n_samples):
    """Replay sampled packages of the given items alone on the oracle and
    compare their step counts with the device's."""
    for k in k_items:
        s = specs[k]
        n = s["n_packages"]
        pids = np.concatenate([[0, n - 1], rng.integers(0, n, n_samples)])
        got = steps_dev[starts[k] + torch.from_numpy(pids).cuda()].cpu().numpy().view(np.uint32)
        for pid, g in zip(pids, got):
            spec = dict(s, cloud=ci, pid_offset=int(pid), n_packages=1)
            _, _, so = oracle_item(w, ci, spec)
            assert g == so[0], (k, pid)


def _conserved(tally, stats, specs, lens):
    """sum(tally of the item) + escaped == emitted for every item, on the device."""
    st = stats.cpu().numpy()
    off = 0
    for k, (s, n) in enumerate(zip(specs, lens)):
        assert int(tally[off:off + n].sum().item()) + int(st[k, 0]) == int(st[k, 3]), k
        off += n
    assert np.all(st[:, 1] == 0)


def test_full_size_octree_sampled_parity():
    """The 4.4e6-cell octree, 64 nu x (1e6 background + 1e6 point-source
    packages) in one launch, as the octree bench times it."""
    w = I.config_c3()
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    specs = []
    for src, npk in ((0, w.n_bg[0]), (1, w.n_ps[0])):
        for f in range(nf):
            specs.append(dict(source=src, freq=f, n_packages=npk, tally_offset=len(specs) * cl.n_cells))
    total = sum(s["n_packages"] for s in specs)
    tally = torch.zeros(len(specs) * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    steps = torch.zeros(total, dtype=torch.int32, device="cuda")
    ctx.simulate(ctx.items(specs), tally, stats, steps)
    torch.cuda.synchronize()
    _conserved(tally, stats, specs, [cl.n_cells] * len(specs))
    assert int(stats[:, 2].sum().item()) == int(steps.to(torch.int64).sum().item())
    starts = np.concatenate([[0], np.cumsum([s["n_packages"] for s in specs])])
    _sample_and_check(w, 0, specs, (0, 37, nf + 5, 2 * nf - 1), steps, starts, np.random.default_rng(3), 6)
    # a contiguous package range of one item: counters bit-exact
    sub = [dict(source=1, freq=30, pid_offset=400_000, n_packages=3000, tally_offset=0)]
    t, st, _ = run_gpu(ctx, sub, cl.n_cells, want_steps=False)
    t_o, st_o, _ = oracle_item(w, 0, sub[0])
    np.testing.assert_array_equal(t, t_o)
    assert st[0][0] == st_o["escaped"] and st[0][3] == st_o["emitted"]


def test_full_size_uneven_batch_sampled_parity():
    """The 64-cloud batch (32^3-128^3, 32 nu, background + point sources) in
    one launch, as its bench times it; sampled packages of four clouds."""
    w = I.config_c5()
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    specs, lens, owner, off = [], [], [], 0
    for ci, cl in enumerate(w.clouds):
        for src, npk in ((0, w.n_bg[ci]), (1, w.n_ps[ci])):
            for f in range(nf):
                specs.append(dict(cloud=ids[ci], source=src, freq=f, n_packages=npk, tally_offset=off))
                lens.append(cl.n_cells)
                owner.append(ci)
                off += cl.n_cells
    total = sum(s["n_packages"] for s in specs)
    tally = torch.zeros(off, dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    steps = torch.zeros(total, dtype=torch.int32, device="cuda")
    ctx.simulate(ctx.items(specs), tally, stats, steps)
    torch.cuda.synchronize()
    _conserved(tally, stats, specs, lens)
    starts = np.concatenate([[0], np.cumsum([s["n_packages"] for s in specs])])
    rng = np.random.default_rng(4)
    for ci in (0, 17, 40, 63):
        ks = [k for k in range(len(specs)) if owner[k] == ci]
        _sample_and_check(w, ci, specs, (ks[3], ks[nf + 20]), steps, starts, rng, 3)


def _deep_octree(ell):
    """2^3 root grid with one path refined down to the deepest level the
    library accepts (16 levels), plus a second octet per level: packages near
    the path climb and descend through all 15 ancestor levels."""
    rho = np.random.default_rng(12).uniform(0.5, 2.0, (2, 2, 2)).astype(np.float32)
    cl = I.regular(rho, ell=ell)
    c, octant = 7, 7
    for level in range(15):
        extra = cl.level_start[-2] + ((c - cl.level_start[-2] + 3) % (cl.level_start[-1] - cl.level_start[-2]))
        cl = I.refine_cells(cl, sorted({int(c), int(extra)}))
        c = int(cl.child[c]) + octant
        octant = 7 - octant
    return cl


@pytest.mark.parametrize("source", [0, 1, 2])
def test_deepest_octree_bit_exact(source):
    base = I.config_c3(root_n=6, max_refine=1, n_freq=8)
    cl = _deep_octree(base.clouds[0].ell)
    assert cl.n_levels == 16
    w = I.Workload("deep16", [cl], base.dust, [base.bg_I[0]], [np.array([[1.6667, 1.6666, 1.6668]])],
                   [base.ps_L[0][:1]], [0], [0], seed=3)
    ctx, ids = gpu_context(w)
    f = 4                                   # tau_abs ~ 1, tau_sca ~ 0.2 per root cell
    n = cl.leaves().size if source == 2 else 4000
    spec = dict(cloud=ids[0], source=source, freq=f, n_packages=n, tally_offset=0)
    dw = None
    if source == 2:
        dw = np.random.default_rng(2).integers(1, 2 ** 31, cl.leaves().size).astype(np.uint64)
        spec["dust_w"] = torch.from_numpy(dw.view(np.int64)).cuda()
    t, st, sp = run_gpu(ctx, [spec], cl.n_cells)
    spec.pop("dust_w", None)
    to, sto, so = oracle_item(w, 0, dict(spec, cloud=0), dust_w=dw)
    np.testing.assert_array_equal(t, to)
    assert st[0][0] == sto["escaped"] and st[0][2] == sto["steps"] and st[0][3] == sto["emitted"]
    np.testing.assert_array_equal(sp, so)
    # refined levels were crossed; the point source (placed on the refined
    # path) and dust (emitted from every leaf) reach the deepest level
    assert t[cl.level_start[2]:].sum() > 0
    if source != 0:
        assert t[cl.level_start[15]:cl.level_start[16]].sum() > 0


def _host_mem_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def test_grid_of_2_30_cells_bit_exact():
    """A 1024^3 regular grid (2^30 cells: 4 GiB of cell words, 8 GiB of
    counters per item, so byte offsets past 2^32 everywhere): background and
    point-source packages give the oracle's counters bit for bit."""
    if _host_mem_gb() < 64 or torch.cuda.get_device_properties(0).total_memory < 64 * 2 ** 30:
        pytest.skip("needs 64 GiB of host and device memory")
    n = 1024
    rho = np.random.default_rng(7).random(n ** 3, dtype=np.float32)
    rho += np.float32(0.5)
    cl = I.regular(rho.reshape(n, n, n), ell=1.0)
    del rho
    dust = I.Dust(np.array([1e14]), np.array([2e-3]), np.array([1e-3]), np.array([0.4]))
    w = I.Workload("big", [cl], dust, [np.array([1.0])], [np.array([[511.3, 300.7, 700.2]])], [np.ones((1, 1))],
                   [0], [0], seed=17)
    ctx, ids = gpu_context(w)
    for src in (0, 1):
        spec = dict(source=src, freq=0, n_packages=2000, tally_offset=0)
        t, st, sp = run_gpu(ctx, [spec], cl.n_cells)
        to, sto, so = oracle_item(w, 0, dict(spec, cloud=0))
        assert np.array_equal(t, to)
        assert st[0][0] == sto["escaped"] and st[0][2] == sto["steps"] and st[0][3] == sto["emitted"]
        np.testing.assert_array_equal(sp, so)
        # packages reach the far corner of the grid (cell indices near 2^30)
        assert t[(n ** 3) * 3 // 4:].sum() > 0
        del t, to
    ctx.close()
