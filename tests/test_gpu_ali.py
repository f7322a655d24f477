"""Accelerated lambda iteration (diagonal operator) on the GPU: the self
counters are bit-identical to the oracle's, the ALI temperature update
agrees with the FP64 oracle within 1e-4, and the accelerated iteration
reaches the plain iteration's fixed point in no more iterations."""
import numpy as np
import pytest

from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context, oracle_grid, oracle_item

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_self_counters_bit_exact():
    w = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0, tau_peak_1um=60.0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    leaf = cl.leaves()
    rng = np.random.default_rng(2)
    dw = rng.integers(0, 2 ** 31, leaf.size).astype(np.uint64)
    dw_t = torch.from_numpy(dw.view(np.int64)).cuda()
    specs = [dict(source=2, freq=f, n_packages=leaf.size, dust_w=dw_t, tally_offset=k * cl.n_cells)
             for k, f in enumerate((10, 40, 60))]
    specs.append(dict(source=0, freq=40, n_packages=2000, tally_offset=3 * cl.n_cells))
    tally = torch.zeros(4 * cl.n_cells, dtype=torch.int64, device="cuda")
    selft = torch.zeros_like(tally)
    stats = torch.zeros((4, 4), dtype=torch.int64, device="cuda")
    ctx.simulate(ctx.items(specs), tally, stats, self_tally=selft)
    torch.cuda.synchronize()
    t, sf = tally.cpu().numpy(), selft.cpu().numpy()
    for k, s in enumerate(specs):
        so = np.zeros(cl.n_cells, np.int64)
        from parity_helpers import kappa_root
        import oracle
        ka, ks = kappa_root(w.dust, s["freq"], cl.ell)
        kw = dict(source=s["source"], kabs=ka, ksca=ks, g=np.float32(w.dust.g[s["freq"]]), seed=w.seed,
                  freq=s["freq"], n_packages=s["n_packages"], self_tally=so)
        if s["source"] == 2:
            kw.update(leaf=leaf, dust_w=dw, n_per_cell=1)
        to = oracle.trace(oracle_grid(cl), **kw)[0]
        np.testing.assert_array_equal(t[k * cl.n_cells:(k + 1) * cl.n_cells], to)
        np.testing.assert_array_equal(sf[k * cl.n_cells:(k + 1) * cl.n_cells], so)
    assert sf[3 * cl.n_cells:].sum() == 0          # background packages have no home cell


def test_ali_temperature_kernel_matches_oracle():
    w = I.config_c3(root_n=6, max_refine=2, threshold=3.0, n_freq=24)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    nu, kabs = w.dust.nu, w.dust.kabs
    leaf = cl.leaves()
    rng = np.random.default_rng(4)
    T_old = rng.uniform(5, 400, cl.n_cells).astype(np.float32)
    T_star = rng.uniform(5, 400, cl.n_cells)
    beta = rng.uniform(0, 1.2, cl.n_cells)
    A = np.array([P.emission_integral(t, nu, kabs) for t in T_star])
    A_self = np.minimum(beta * np.array([P.emission_integral(float(t), nu, kabs) for t in T_old]), 0.95 * A)
    Td = torch.from_numpy(T_old).cuda()
    ctx.update_temperature_ali(ids[0], torch.from_numpy(A).cuda(), torch.from_numpy(A_self).cuda(), Td)
    Tg = Td.cpu().numpy()
    To = np.array([P.temperature_ali(A[c], A_self[c], float(T_old[c]), nu, kabs) for c in leaf])
    np.testing.assert_allclose(Tg[leaf], To, rtol=1e-4)


def test_ali_iteration_converges_to_plain_fixed_point():
    w = I.config_c3(root_n=8, max_refine=2, sigma=1.5, threshold=4.0, tau_peak_1um=300.0, n_freq=24,
                    L_bol=3e36, side_pc=0.1, n_bg=20000, n_ps=20000)
    cl = w.clouds[0]
    res = {}
    for ali in (False, True):
        ctx, ids = gpu_context(w)
        T = torch.zeros(cl.n_cells, dtype=torch.float32, device="cuda")
        r = ctx.iterate(ids[0], T, n_background=w.n_bg[0], n_point=w.n_ps[0], n_per_cell=1, max_iter=60,
                        dT_tol=0.05, ali=ali)
        res[ali] = (r, T.cpu().numpy())
        ctx.close()
    (rp, Tp), (ra, Ta) = res[False], res[True]
    assert rp["converged"] and ra["converged"]
    assert ra["iterations"] <= rp["iterations"]
    leaf = cl.leaves()
    assert np.abs(Ta[leaf] - Tp[leaf]).max() < 1.0
