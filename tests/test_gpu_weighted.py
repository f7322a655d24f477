"""Emission-weighted dust sampling on the GPU: the allocation (packages per
cell, weights, prefix) is bit-identical to the oracle's from the same uniform
weights, and tracing weighted dust packages gives bit-identical counters."""
import numpy as np
import pytest

import oracle
from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, kappa_root, oracle_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _setup(n_total, cap):
    w = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0, tau_peak_1um=40.0, n_freq=8)
    cl = w.clouds[0]
    leaf = cl.leaves()
    rng = np.random.default_rng(9)
    T = rng.uniform(8, 300, leaf.size)
    V = P.cell_volumes(oracle_grid(cl), cl.ell)
    nf = len(w.dust.nu)
    us, es = [], []
    for f in range(nf):
        L = P.dust_luminosity(T, cl.rho[leaf], V[leaf], w.dust.kabs[f], w.dust.nu[f])
        u, e = P.dust_weights(L, 1)
        us.append(u); es.append(e)
    return w, cl, leaf, np.array(us), np.array(es)


@pytest.mark.parametrize("n_total,cap", [(20000, 50), (5000, 10000), (3, 1)])
def test_weighted_allocation_bit_exact(n_total, cap):
    w, cl, leaf, U, E = _setup(n_total, cap)
    nf, nl = U.shape
    ctx, ids = gpu_context(w)
    u_d = torch.from_numpy(U.view(np.int64)).cuda()
    e_d = torch.from_numpy(E).cuda()
    out = torch.zeros((nf, 2 * nl + 1), dtype=torch.int64, device="cuda")
    eo = torch.zeros(nf, dtype=torch.float64, device="cuda")
    ctx.dust_weighted(ids[0], u_d, e_d, n_total, cap, out, eo)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    ge = eo.cpu().numpy()
    for f in range(nf):
        n, pref, W, e = P.weighted_dust_sampling(U[f], E[f], n_total, cap)
        np.testing.assert_array_equal(got[f, :nl], W)
        np.testing.assert_array_equal(got[f, nl:], pref)
        assert ge[f] == e or abs(ge[f] / e - 1) < 1e-15


def test_weighted_dust_tracing_bit_exact():
    """Weighted dust packages (allocation made by the oracle, uploaded as the
    tracer's input) give the oracle's counters, stats and step counts."""
    w, cl, leaf, U, E = _setup(0, 0)
    nf, nl = U.shape
    ctx, ids = gpu_context(w)
    n_total, cap = 6 * nl, 40
    alloc = np.zeros((nf, 2 * nl + 1), np.uint64)
    for f in range(nf):
        _, pref, W, _ = P.weighted_dust_sampling(U[f], E[f], n_total, cap)
        alloc[f, :nl], alloc[f, nl:] = W, pref
    out = torch.from_numpy(alloc.view(np.int64)).cuda()
    specs = []
    for k, f in enumerate((1, 4, 7)):
        specs.append(dict(source=2, freq=f, n_packages=int(alloc[f, 2 * nl]), dust_w=out[f], weighted=True,
                          tally_offset=k * cl.n_cells))
    tally = torch.zeros(3 * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((3, 4), dtype=torch.int64, device="cuda")
    steps = torch.zeros(sum(s["n_packages"] for s in specs), dtype=torch.int32, device="cuda")
    ctx.simulate(ctx.items(specs), tally, stats, steps)
    torch.cuda.synchronize()
    t = tally.cpu().numpy()
    st = stats.cpu().numpy()
    sp = steps.cpu().numpy().view(np.uint32)
    off = 0
    for k, s in enumerate(specs):
        f = s["freq"]
        ka, ks = kappa_root(w.dust, f, cl.ell)
        to, sto, so = oracle.trace(oracle_grid(cl), source=2, kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed,
                                   freq=f, n_packages=s["n_packages"], leaf=leaf, dust_w=alloc[f, :nl],
                                   dust_prefix=alloc[f, nl:], want_steps=True)
        np.testing.assert_array_equal(t[k * cl.n_cells:(k + 1) * cl.n_cells], to)
        assert st[k][0] == sto["escaped"] and st[k][3] == sto["emitted"]
        np.testing.assert_array_equal(sp[off:off + s["n_packages"]], so)
        off += s["n_packages"]


def test_reweight_bit_exact():
    """A frozen allocation re-weighted at new temperatures equals the oracle."""
    w, cl, leaf, U, E = _setup(0, 0)
    nf, nl = U.shape
    ctx, ids = gpu_context(w)
    alloc = np.zeros((nf, 2 * nl + 1), np.uint64)
    for f in range(nf):
        _, pref, W, _ = P.weighted_dust_sampling(U[f], E[f], 5 * nl, 30)
        alloc[f, :nl], alloc[f, nl:] = W, pref
    out = torch.from_numpy(alloc.view(np.int64).copy()).cuda()
    eo = torch.zeros(nf, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(21)
    T2 = rng.uniform(8, 300, nl)
    V = P.cell_volumes(oracle_grid(cl), cl.ell)
    U2, E2 = [], []
    for f in range(nf):
        u, e = P.dust_weights(P.dust_luminosity(T2, cl.rho[leaf], V[leaf], w.dust.kabs[f], w.dust.nu[f]), 1)
        U2.append(u); E2.append(e)
    U2, E2 = np.array(U2), np.array(E2)
    ctx.dust_reweight(ids[0], torch.from_numpy(U2.view(np.int64)).cuda(), torch.from_numpy(E2).cuda(), out, eo)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    ge = eo.cpu().numpy()
    np.testing.assert_array_equal(got[:, nl:], alloc[:, nl:])         # counts kept
    for f in range(nf):
        W, e = P.weighted_dust_reweight(U2[f], E2[f], alloc[f, nl:])
        np.testing.assert_array_equal(got[f, :nl], W)
        assert ge[f] == e or abs(ge[f] / e - 1) < 1e-15


def _dust_absorbed(ctx, cid, cl, T, nf, weighted, n_total, cap):
    """Absorbed power from dust emission only (fixed T), one pass."""
    leaf = cl.leaves()
    nl = leaf.size
    u = torch.zeros((nf, nl), dtype=torch.int64, device="cuda")
    e = torch.zeros(nf, dtype=torch.float64, device="cuda")
    ctx.dust_emission(cid, T, u, e, n_per_cell=1)
    tally = torch.zeros(nf * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((nf, 4), dtype=torch.int64, device="cuda")
    if weighted:
        out = torch.zeros((nf, 2 * nl + 1), dtype=torch.int64, device="cuda")
        ew = torch.zeros(nf, dtype=torch.float64, device="cuda")
        ctx.dust_weighted(cid, u, e, n_total, cap, out, ew)
        torch.cuda.synchronize()
        counts = out[:, 2 * nl].cpu().numpy()
        specs = [dict(source=2, freq=f, n_packages=int(counts[f]), dust_w=out[f], weighted=True, iteration=1,
                      tally_offset=f * cl.n_cells) for f in range(nf)]
        e_use = ew
    else:
        per = max(1, n_total // nl)
        u2 = torch.zeros((nf, nl), dtype=torch.int64, device="cuda")
        ctx.dust_emission(cid, T, u2, e, n_per_cell=per)
        specs = [dict(source=2, freq=f, n_packages=nl * per, dust_w=u2[f], n_per_cell=per, iteration=1,
                      tally_offset=f * cl.n_cells) for f in range(nf)]
        e_use = e
    ctx.simulate(ctx.items(specs), tally, stats)
    A = torch.zeros(cl.n_cells, dtype=torch.float64, device="cuda")
    ctx.absorbed_power(cid, tally, cl.n_cells, e_use, A)
    torch.cuda.synchronize()
    return A.cpu().numpy(), int(stats[:, 3].sum().item() > 0)


def test_weighted_sampling_lowers_noise_for_equal_budget():
    """Two seeds, same temperatures with a hot core: the seed-to-seed spread of
    the absorbed dust power (cells heated most by the dust) is smaller with
    emission weighting than with the same number of uniform packages."""
    w = I.config_c2(n=24, n_freq=16, n_packages=0, tau_1um=30.0)
    cl = w.clouds[0]
    n = 24
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r2 = ((i - 11.5) ** 2 + (j - 11.5) ** 2 + (k - 11.5) ** 2).ravel()
    T_host = (15.0 + 250.0 * np.exp(-r2 / 8.0)).astype(np.float32)
    T = torch.from_numpy(T_host).cuda()
    nf = len(w.dust.nu)
    budget = 2 * cl.n_cells
    res = {}
    from paper_1812_06632_gb300 import soc
    for weighted in (False, True):
        As = []
        for seed in (11, 12):
            ctx = soc.Context(0, seed)
            ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
            cid = ctx.grid_upload(cl)
            As.append(_dust_absorbed(ctx, cid, cl, T, nf, weighted, budget, 200)[0])
            ctx.close()
        res[weighted] = As
    # cells around the hot core (chosen by geometry, not by a noisy sample)
    hot = np.flatnonzero(r2 <= 20.0)
    def spread(As):
        a, b = As[0][hot], As[1][hot]
        return float(np.sqrt(np.mean(((a - b) / (0.5 * (a + b))) ** 2)))
    s_uni, s_w = spread(res[False]), spread(res[True])
    # the same field in expectation
    m_uni = 0.5 * (res[False][0][hot].mean() + res[False][1][hot].mean())
    m_w = 0.5 * (res[True][0][hot].mean() + res[True][1][hot].mean())
    assert abs(m_w / m_uni - 1) < 0.05, (m_w, m_uni)
    assert s_w < 0.8 * s_uni, (s_w, s_uni)


def test_iterate_weighted_converges():
    """Dust iterations with emission weighting (cap 10000 packages per cell, as
    in the paper's Sect. 4 test) converge with frozen random numbers and reach
    the temperatures of a uniform run with 512x the packages.  A uniform run
    with the weighted run's budget is biased low by its noise (few hits per
    cell through the concave T(A)), far more than the weighted one."""
    w = I.config_c3(root_n=8, max_refine=2, sigma=1.5, threshold=4.0, tau_peak_1um=200.0, n_freq=16,
                    L_bol=3e36, side_pc=0.1, n_bg=20000, n_ps=20000)
    cl = w.clouds[0]
    leaf = cl.leaves()
    res = {}
    for mode, kw in (("uniform", dict(n_per_cell=2)), ("reference", dict(n_per_cell=1024)),
                     ("weighted", dict(n_weighted=2 * leaf.size, weighted_cap=10000))):
        ctx, ids = gpu_context(w)
        T = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
        r = ctx.iterate(ids[0], T, n_background=w.n_bg[0], n_point=w.n_ps[0], max_iter=20, dT_tol=0.1, **kw)
        assert r["converged"], mode
        res[mode] = float(T.cpu().numpy()[leaf].mean())
        ctx.close()
    err_w = abs(res["weighted"] / res["reference"] - 1)
    err_u = abs(res["uniform"] / res["reference"] - 1)
    assert err_w < 0.02 and err_u > 3 * err_w, res
