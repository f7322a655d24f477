"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tracer: the int64 fixed-point counters, escaped / emitted weights and the
per-package step counts must be bit-identical to the oracle's for the same
seeded inputs.  FP64 normalisation: absorbed power within 1e-14 relative;
temperatures within 1e-4 relative of the oracle's Brent root; dust weights
within one fixed-point unit (FP64 exp of two libraries may differ in the last
bit).
"""
import numpy as np
import pytest

import oracle
from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import W_UNIT, gpu_context, oracle_grid, oracle_item, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare_item(w, ci, spec, tally, stats_row, steps, n_cells, offset=0, dust_w=None):
    t_o, st_o, steps_o = oracle_item(w, ci, spec, dust_w=dust_w)
    np.testing.assert_array_equal(tally[offset:offset + n_cells], t_o)
    assert stats_row[0] == st_o["escaped"]
    assert stats_row[1] == st_o["capped"]
    assert stats_row[2] == st_o["steps"]
    assert stats_row[3] == st_o["emitted"]
    if steps is not None:
        np.testing.assert_array_equal(steps, steps_o)
    # exact conservation on the GPU side by itself
    assert int(tally[offset:offset + n_cells].sum()) + int(stats_row[0]) == int(stats_row[3])


def test_c1_uniform_cube_bit_exact():
    """32^3 uniform cube, tau = 1 centre-to-edge, albedo 0.5, 1e5 packages."""
    w = I.config_c1()
    ctx, ids = gpu_context(w)
    cl = w.clouds[0]
    spec = dict(source=0, freq=0, n_packages=100_000)
    tally, stats, steps = run_gpu(ctx, [spec], cl.n_cells)
    _compare_item(w, 0, spec, tally, stats[0], steps, cl.n_cells)


def test_lognormal_multifrequency_batch_bit_exact():
    """24^3 lognormal cloud, 6 frequencies spanning tau 1e-4..1e2, HG g=0.5,
    ragged package counts, all in one launch."""
    w = I.config_c2(n=24, n_freq=64, n_packages=0)
    ctx, ids = gpu_context(w)
    cl = w.clouds[0]
    freqs = [5, 20, 35, 45, 55, 63]
    specs = [dict(source=0, freq=f, n_packages=3000 + 37 * k, tally_offset=k * cl.n_cells)
             for k, f in enumerate(freqs)]
    tally, stats, steps = run_gpu(ctx, specs, len(specs) * cl.n_cells)
    off = 0
    for k, s in enumerate(specs):
        n = s["n_packages"]
        _compare_item(w, 0, s, tally, stats[k], steps[off:off + n], cl.n_cells, offset=k * cl.n_cells)
        off += n


def _dust_weights(w, cl, f, n_per_cell=1):
    T = 8.0 + 40.0 * (cl.rho / cl.rho.max())
    leaf = cl.leaves()
    L = P.dust_luminosity(T[leaf], cl.rho[leaf], P.cell_volumes(oracle_grid(cl), cl.ell)[leaf],
                          w.dust.kabs[f], w.dust.nu[f])
    return P.dust_weights(L, n_per_cell)[0]


def test_octree_background_point_dust_one_launch_bit_exact():
    """Octree (root 8^3, 3 refinement levels), 3 point sources + background +
    dust re-emission (2 packages per leaf) mixed in one launch."""
    w = I.config_c3(root_n=8, max_refine=3, sigma=2.0, threshold=3.0, tau_peak_1um=30.0)
    cl = w.clouds[0]
    assert cl.n_levels == 4
    ctx, ids = gpu_context(w)
    f_bg, f_ps, f_d = 30, 44, 12
    dw = _dust_weights(w, cl, f_d, 2)
    dw_t = torch.from_numpy(dw.view(np.int64)).cuda()
    nl = cl.leaves().size
    specs = [dict(source=0, freq=f_bg, n_packages=4001, tally_offset=0),
             dict(source=1, freq=f_ps, n_packages=3007, tally_offset=cl.n_cells),
             dict(source=2, freq=f_d, n_packages=2 * nl, n_per_cell=2, dust_w=dw_t,
                  tally_offset=2 * cl.n_cells)]
    tally, stats, steps = run_gpu(ctx, specs, 3 * cl.n_cells)
    off = 0
    for k, s in enumerate(specs):
        n = s["n_packages"]
        _compare_item(w, 0, s, tally, stats[k], steps[off:off + n], cl.n_cells, offset=k * cl.n_cells,
                      dust_w=dw if s["source"] == 2 else None)
        off += n


def test_two_clouds_uneven_batch_bit_exact():
    w = I.config_c5(n_clouds=2, n_freq=4, sizes=[16, 24], base_packages=2000)
    ctx, ids = gpu_context(w)
    specs, offs, off = [], [], 0
    for ci, cl in enumerate(w.clouds):
        for src in (0, 1):
            for f in (1, 3):
                specs.append(dict(cloud=ids[ci], source=src, freq=f, n_packages=1500 + 11 * ci,
                                  tally_offset=off))
                offs.append((ci, off))
                off += cl.n_cells
    tally, stats, steps = run_gpu(ctx, specs, off)
    p = 0
    for k, s in enumerate(specs):
        ci, o = offs[k]
        n = s["n_packages"]
        _compare_item(w, ci, s, tally, stats[k], steps[p:p + n], w.clouds[ci].n_cells, offset=o)
        p += n


@pytest.mark.parametrize("tpb,bps,chunk,refill,scatter", [(32, 0, 1, 1, 1), (128, 2, 7, 4, 8), (256, 0, 64, 16, 32),
                                                            (64, 1, 3, 32, 3), (256, 4, 16, 8, 16)])
def test_launch_shape_does_not_change_results(tpb, bps, chunk, refill, scatter):
    w = I.config_c2(n=20, n_freq=64, n_packages=0)
    ctx, ids = gpu_context(w)
    cl = w.clouds[0]
    specs = [dict(source=0, freq=f, n_packages=2500, tally_offset=k * cl.n_cells)
             for k, f in enumerate((10, 50, 63))]
    ref = run_gpu(ctx, specs, 3 * cl.n_cells)
    ctx.set_launch(tpb, bps, chunk)
    ctx.set_refill(refill)
    ctx.set_scatter_batch(scatter)
    got = run_gpu(ctx, specs, 3 * cl.n_cells)
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_package_subrange_and_empty_items():
    w = I.config_c2(n=16, n_freq=64, n_packages=0)
    ctx, ids = gpu_context(w)
    cl = w.clouds[0]
    specs = [dict(source=0, freq=40, n_packages=0, tally_offset=0),
             dict(source=0, freq=40, pid_offset=12345, n_packages=777, tally_offset=0),
             dict(source=0, freq=40, n_packages=0, tally_offset=cl.n_cells)]
    tally, stats, steps = run_gpu(ctx, specs, 2 * cl.n_cells)
    assert np.all(stats[0] == 0) and np.all(stats[2] == 0)
    assert np.all(tally[cl.n_cells:] == 0)
    _compare_item(w, 0, specs[1], tally, stats[1], steps, cl.n_cells)


def test_paper_link_encoding_upload_gives_same_counters():
    w = I.config_c3(root_n=6, max_refine=2, threshold=3.0)
    cl = w.clouds[0]
    from paper_1812_06632_gb300 import soc
    ctx_a, _ = gpu_context(w)
    ctx_b = soc.Context(0, w.seed)
    ctx_b.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    cid = ctx_b.grid_upload(cl, paper_encoding=True)
    ctx_b.sources_upload(cid, w.bg_I[0], w.ps_pos[0], w.ps_L[0])
    specs = [dict(source=0, freq=40, n_packages=3000)]
    a = run_gpu(ctx_a, specs, cl.n_cells)
    b = run_gpu(ctx_b, specs, cl.n_cells)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_step_cap_matches_oracle():
    cl = I.regular(np.ones((8, 8, 8), np.float32))
    w = I.Workload("cap", [cl], I.Dust(np.array([1e14]), np.array([0.01]), np.array([3.0]), np.array([0.2])),
                   [np.array([1.0])], [None], [None], [500], [0], seed=3)
    ctx, ids = gpu_context(w)
    ctx.set_max_steps(5)
    spec = dict(source=0, freq=0, n_packages=500, max_steps=5)
    tally, stats, steps = run_gpu(ctx, [dict(source=0, freq=0, n_packages=500)], cl.n_cells)
    assert stats[0][1] > 0 and steps.max() == 5
    _compare_item(w, 0, spec, tally, stats[0], steps, cl.n_cells)


def test_step_cap_on_an_octree_matches_oracle():
    """Capped packages on an octree, where a crossing into a refined cell
    leaves the descent to the warp's descent phase: the cap still ends each
    package after the same steps, in the same leaf, as the oracle."""
    w = I.config_c3(root_n=8, max_refine=3, threshold=3.0, tau_peak_1um=80.0, n_freq=8)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    ctx.set_max_steps(7)
    for src in (0, 1):
        spec = dict(source=src, freq=5, n_packages=3000)
        tally, stats, steps = run_gpu(ctx, [spec], cl.n_cells)
        assert stats[0][1] > 0 and steps.max() == 7
        _compare_item(w, 0, dict(spec, max_steps=7), tally, stats[0], steps, cl.n_cells)


@pytest.mark.parametrize("case", ["one_cell", "empty_density", "opaque"])
def test_degenerate_grids(case):
    if case == "one_cell":
        cl = I.regular(np.ones((1, 1, 1), np.float32))
        kabs, ksca = 0.7, 0.9
    elif case == "empty_density":
        cl = I.regular(np.zeros((5, 6, 7), np.float32))
        kabs, ksca = 1.0, 1.0
    else:
        cl = I.regular(np.full((6, 6, 6), 1e4, np.float32))
        kabs, ksca = 1.0, 0.5
    w = I.Workload(case, [cl], I.Dust(np.array([1e14]), np.array([kabs]), np.array([ksca]), np.array([0.3])),
                   [np.array([1.0])], [np.array([[cl.nx / 2 + 0.1, cl.ny / 2 - 0.2, cl.nz / 2 + 0.05]])],
                   [np.ones((1, 1))], [2000], [2000], seed=9)
    ctx, ids = gpu_context(w)
    for src in (0, 1):
        spec = dict(source=src, freq=0, n_packages=2000)
        tally, stats, steps = run_gpu(ctx, [spec], cl.n_cells)
        _compare_item(w, 0, spec, tally, stats[0], steps, cl.n_cells)
        if case == "empty_density":
            assert tally.sum() == 0 and stats[0][0] == stats[0][3]


# ----------------------------------------------------------------------------
# FP64 steps: absorbed power, temperature, dust weights
# ----------------------------------------------------------------------------
def _thin_workload():
    w = I.config_c3(root_n=8, max_refine=2, sigma=1.5, threshold=3.0, tau_peak_1um=20.0, n_freq=24)
    return w


def test_absorbed_power_and_temperature_match_oracle():
    w = _thin_workload()
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    N = 3000
    specs = [dict(source=0, freq=f, n_packages=N, tally_offset=f * cl.n_cells) for f in range(nf)]
    tally, stats, _ = run_gpu(ctx, specs, nf * cl.n_cells, want_steps=False)
    # the counters themselves are pinned by the tracer tests; check two frequencies
    for f in (3, 17):
        t_o = oracle_item(w, 0, specs[f])[0]
        np.testing.assert_array_equal(tally[f * cl.n_cells:(f + 1) * cl.n_cells], t_o)
    # counters for the integral: seeded, made on the host (both sides take them)
    tal2 = np.random.default_rng(31).integers(0, 2 ** 36, (nf, cl.n_cells)).astype(np.int64)
    tal2[:, ::7] = 0
    e = P.background_package_energy(w.bg_I[0], cl.nx, cl.ny, cl.nz, cl.ell, N)
    np.testing.assert_allclose(ctx.package_energy(ids[0], 0, N), e, rtol=1e-15)
    A_o = P.absorbed_power(tal2, e, w.dust.nu, cl.rho, P.cell_volumes(oracle_grid(cl), cl.ell))
    t_dev = torch.from_numpy(tal2.ravel()).cuda()
    e_dev = torch.from_numpy(e).cuda()
    A = torch.zeros(cl.n_cells, dtype=torch.float64, device="cuda")
    ctx.absorbed_power(ids[0], t_dev, cl.n_cells, e_dev, A)
    T = torch.full((cl.n_cells,), 2.7, dtype=torch.float32, device="cuda")
    dT = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.update_temperature(ids[0], A, T, dT)
    torch.cuda.synchronize()
    A_g = A.cpu().numpy()
    leaf = cl.leaves()
    np.testing.assert_allclose(A_g[leaf], A_o[leaf], rtol=1e-14, atol=0)
    T_o = P.temperatures(A_o[leaf], w.dust.nu, w.dust.kabs)
    T_g = T.cpu().numpy()[leaf]
    np.testing.assert_allclose(T_g, T_o, rtol=1e-4)
    assert abs(dT.item() - np.abs(T_g.astype(np.float64) - 2.7).max()) < 1e-6


def test_temperature_extremes_and_closed_form_field():
    """A = 0 -> 2.7 K; huge A -> 3000 K; A from a diluted blackbody field."""
    w = _thin_workload()
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    nu, kabs = w.dust.nu, w.dust.kabs
    leaf = cl.leaves()
    Tstar = np.geomspace(3.0, 2500.0, leaf.size)
    A_host = np.zeros(cl.n_cells)
    A_host[leaf] = [P.emission_integral(t, nu, kabs) for t in Tstar]
    A_host[leaf[:3]] = [0.0, 1e-300, 1e300]
    A = torch.from_numpy(A_host).cuda()
    T = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
    ctx.update_temperature(ids[0], A, T)
    Tg = T.cpu().numpy()[leaf]
    assert Tg[0] == np.float32(2.7) and Tg[1] == np.float32(2.7) and Tg[2] == np.float32(3000.0)
    np.testing.assert_allclose(Tg[3:], Tstar[3:], rtol=1e-4)


def test_dust_emission_weights_match_oracle():
    w = _thin_workload()
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    T_host = (8.0 + 60.0 * (cl.rho / cl.rho.max())).astype(np.float32)
    T = torch.from_numpy(T_host).cuda()
    leaf = cl.leaves()
    W = torch.zeros((nf, leaf.size), dtype=torch.int64, device="cuda")
    e = torch.zeros(nf, dtype=torch.float64, device="cuda")
    ctx.dust_emission(ids[0], T, W, e, n_per_cell=3)
    torch.cuda.synchronize()
    Wg = W.cpu().numpy().view(np.uint64)
    eg = e.cpu().numpy()
    V = P.cell_volumes(oracle_grid(cl), cl.ell)
    for f in range(nf):
        L = P.dust_luminosity(T_host[leaf].astype(np.float64), cl.rho[leaf], V[leaf], w.dust.kabs[f], w.dust.nu[f])
        Wo, eo = P.dust_weights(L, 3)
        d = np.abs(Wg[f].astype(np.int64) - Wo.astype(np.int64))
        assert d.max() <= 1, (f, d.max())
        if eo == 0.0:                          # B_nu(T) underflows for every cell
            assert eg[f] == 0.0 and np.all(Wg[f] == 0)
        else:
            assert abs(eg[f] / eo - 1) < 1e-13


def test_iterate_matches_oracle_driven_iteration():
    """soc_iterate (constant sources once, then frozen-seed dust iterations)
    against the same sequence driven step by step with the oracle."""
    w = I.config_c3(root_n=6, max_refine=2, sigma=1.5, threshold=3.0, tau_peak_1um=60.0, n_freq=16,
                    L_bol=3e36, side_pc=0.05)
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    n_bg, n_ps, iters = 1500, 1500, 3
    T = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
    res = ctx.iterate(ids[0], T, n_background=n_bg, n_point=n_ps, n_per_cell=1, max_iter=iters, dT_tol=0.0)
    assert res["iterations"] == iters
    Tg = T.cpu().numpy()
    # oracle
    G = oracle_grid(cl)
    V = P.cell_volumes(G, cl.ell)
    leaf = cl.leaves()
    A_const = np.zeros(cl.n_cells)
    for src, n in ((0, n_bg), (1, n_ps)):
        tal = np.stack([oracle_item(w, 0, dict(source=src, freq=f, n_packages=n))[0] for f in range(nf)])
        e = (P.background_package_energy(w.bg_I[0], cl.nx, cl.ny, cl.nz, cl.ell, n) if src == 0
             else P.point_package_energy(np.asarray(w.ps_L[0]).sum(axis=0), n))
        A_const = P.absorbed_power(tal, e, w.dust.nu, cl.rho, V, A_in=A_const)
    To = np.full(cl.n_cells, 0.0)
    To[leaf] = P.temperatures(A_const[leaf], w.dust.nu, w.dust.kabs)
    for k in range(iters):
        tal = np.zeros((nf, cl.n_cells), np.int64)
        e = np.zeros(nf)
        for f in range(nf):
            L = P.dust_luminosity(To[leaf].astype(np.float32).astype(np.float64), cl.rho[leaf], V[leaf],
                                  w.dust.kabs[f], w.dust.nu[f])
            Wd, e[f] = P.dust_weights(L, 1)
            tal[f] = oracle_item(w, 0, dict(source=2, freq=f, n_packages=leaf.size, iteration=1), dust_w=Wd)[0]
        A = P.absorbed_power(tal, e, w.dust.nu, cl.rho, V, A_in=A_const)
        To[leaf] = P.temperatures(A[leaf], w.dust.nu, w.dust.kabs)
    np.testing.assert_allclose(Tg[leaf], To[leaf], rtol=1e-4)
    assert Tg[leaf].max() > 30.0       # the point sources heat the core


# ----------------------------------------------------------------------------
# full-size workload: 128^3 lognormal, 64 frequencies, 1e6 packages each
# ----------------------------------------------------------------------------
def test_full_size_128cube_64nu_sampled_parity():
    w = I.config_c2()
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx, ids = gpu_context(w)
    N = 1_000_000
    specs = [dict(source=0, freq=f, n_packages=N, tally_offset=f * cl.n_cells) for f in range(nf)]
    tally, stats, steps = run_gpu(ctx, specs, nf * cl.n_cells)
    # exact conservation for every frequency, at full size
    t2 = tally.reshape(nf, cl.n_cells)
    np.testing.assert_array_equal(t2.sum(axis=1) + stats[:, 0], stats[:, 3])
    assert np.all(stats[:, 3] == N * W_UNIT) and np.all(stats[:, 1] == 0)
    assert stats[:, 2].sum() == steps.astype(np.int64).sum()
    # sampled packages, each replayed alone by the oracle
    rng = np.random.default_rng(0)
    for f in (0, 21, 42, 63):
        for pid in np.concatenate([[0, N - 1], rng.integers(0, N, 30)]):
            s = dict(source=0, freq=f, pid_offset=int(pid), n_packages=1)
            t_o, st_o, st1 = oracle_item(w, 0, s)
            assert steps[f * N + pid] == st1[0], (f, pid)
    # a contiguous package range of two frequencies: counters bit-exact
    sub = [dict(source=0, freq=f, pid_offset=250_000, n_packages=4000, tally_offset=k * cl.n_cells)
           for k, f in enumerate((7, 50))]
    ts, ss, _ = run_gpu(ctx, sub, 2 * cl.n_cells, want_steps=False)
    for k, s in enumerate(sub):
        _compare_item(w, 0, s, ts, ss[k], None, cl.n_cells, offset=k * cl.n_cells)
