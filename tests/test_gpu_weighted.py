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
    w, cl, leaf, U, E = _setup(0, 0)
    nf, nl = U.shape
    ctx, ids = gpu_context(w)
    n_total, cap = 6 * nl, 40
    out = torch.zeros((nf, 2 * nl + 1), dtype=torch.int64, device="cuda")
    eo = torch.zeros(nf, dtype=torch.float64, device="cuda")
    ctx.dust_weighted(ids[0], torch.from_numpy(U.view(np.int64)).cuda(), torch.from_numpy(E).cuda(), n_total, cap,
                      out, eo)
    torch.cuda.synchronize()
    host = out.cpu().numpy().view(np.uint64)
    specs = []
    for k, f in enumerate((1, 4, 7)):
        n_pk = int(host[f, 2 * nl])
        specs.append(dict(source=2, freq=f, n_packages=n_pk, dust_w=out[f], weighted=True,
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
                                   freq=f, n_packages=s["n_packages"], leaf=leaf, dust_w=host[f, :nl],
                                   dust_prefix=host[f, nl:], want_steps=True)
        np.testing.assert_array_equal(t[k * cl.n_cells:(k + 1) * cl.n_cells], to)
        assert st[k][0] == sto["escaped"] and st[k][3] == sto["emitted"]
        np.testing.assert_array_equal(sp[off:off + s["n_packages"]], so)
        off += s["n_packages"]
