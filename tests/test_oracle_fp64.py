"""The FP64 Monte Carlo oracle: pinned on its own (exact conservation in
real arithmetic, the brute-force escape probability, the thin-box
background normalisation), then used to state how far the FP32 contract's
counters (the GPU's, bit for bit) are from the same packages traced in FP64
with libm exp/log and real weights (no GPU)."""
import numpy as np
import pytest

import oracle
from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I
from parity_helpers import kappa_root, oracle_grid
from test_oracle_pins import _cube_transmission_quadrature


def _item_kwargs(w, ci, src, f, n):
    cl = w.clouds[ci]
    ka, ks = kappa_root(w.dust, f, cl.ell)
    kw = dict(source=src, kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed, freq=f, n_packages=n)
    if src == 1:
        kw["ps_pos"] = np.asarray(w.ps_pos[ci], np.float64).astype(np.float32)
        kw["ps_cdf"] = P.point_source_cdf(w.ps_L[ci])[f]
    if src == 2:
        leaf = cl.leaves()
        dw = np.random.default_rng(f).integers(1 << 20, 1 << 31, leaf.size).astype(np.uint64)
        kw.update(leaf=leaf, dust_w=dw, n_per_cell=1, n_packages=min(n, leaf.size))
    return kw


def _octree():
    return I.config_c3(root_n=16, max_refine=3, threshold=3.0, n_freq=8, tau_peak_1um=50.0)


@pytest.mark.parametrize("source", [0, 1, 2])
def test_fp64_conserves_energy(source):
    """Absorbed + escaped = emitted, to rounding of real arithmetic."""
    w = _octree()
    kw = _item_kwargs(w, 0, source, 5, 1500)
    t, st, _ = oracle.trace64(oracle_grid(w.clouds[0]), **kw)
    assert st["capped"] == 0
    assert abs(t.sum() + st["escaped"] - st["emitted"]) <= 1e-12 * st["emitted"]
    assert np.all(t >= 0)


@pytest.mark.parametrize("layout", ["1cube", "2cube_refined"])
def test_fp64_brute_force_escape_probability(layout):
    """Albedo 0: escaped fraction = quadrature of exp(-tau(path)) over
    cosine-weighted entry."""
    tau_side = 1.3
    if layout == "1cube":
        cl = I.regular(np.ones((1, 1, 1), np.float32)); k = tau_side
    else:
        cl = I.regular(np.ones((2, 2, 2), np.float32)); k = tau_side / 2
        cl = I.refine_cells(cl, [0, 3, 6])
    N = 200_000
    _, st, _ = oracle.trace64(oracle_grid(cl), source=0, kabs=k, ksca=0.0, seed=21, n_packages=N)
    p_mc = st["escaped"] / st["emitted"]
    assert abs(p_mc - _cube_transmission_quadrature(tau_side)) < 3.5e-3


def test_fp64_thin_box_absorbs_4pi_kappa_I():
    """Optically thin box in an isotropic field I: every cell absorbs
    4 pi kabs I per unit rho V."""
    shape, ell, kabs, I_nu = (3, 4, 5), 2.0, 1e-4, 3.0
    cl = I.regular(np.ones(shape, np.float32), ell=ell)
    N = 100_000
    t, st, _ = oracle.trace64(oracle_grid(cl), source=0, kabs=kabs * ell, ksca=0.0, seed=11, n_packages=N)
    e = P.background_package_energy([I_nu], shape[2], shape[1], shape[0], ell, N)
    A = P.absorbed_power(t[None, :], e, [1.0], cl.rho, P.cell_volumes(oracle_grid(cl), ell))
    ratio = A / (4 * np.pi * kabs * I_nu)
    assert abs(ratio.mean() - 1) < 6e-3


CASES = [("c2_128_bg_low_nu", "c2", 0, 10), ("c2_128_bg_high_nu", "c2", 0, 50),
         ("octree_bg", "oct", 0, 5), ("octree_point", "oct", 1, 5), ("octree_dust", "oct", 2, 5)]


@pytest.mark.parametrize("name,wl,src,f", CASES)
def test_fp32_contract_against_fp64(name, wl, src, f):
    """The same packages traced in the FP32 contract and in FP64.  Bounds
    (measured margins in brackets): at least 97 % of packages take the same
    number of steps (98.2-100 %: a package parts ways only where a rounding
    flips a decision, most often the last step before the weight floor);
    total absorbed energy within 1e-6 of the emitted energy (1e-11-4e-7);
    per-cell counters within 3e-4 in L1 relative to the absorbed total
    (2e-6-1.1e-4; the largest where cells absorb little, since a deposit is
    rounded to whole weight units)."""
    w = I.config_c2(n_packages=0) if wl == "c2" else _octree()
    kw = _item_kwargs(w, 0, src, f, 2000)
    G = oracle_grid(w.clouds[0])
    t32, s32, n32 = oracle.trace(G, want_steps=True, **kw)
    t64, s64, n64 = oracle.trace64(G, want_steps=True, **kw)
    E = s64["emitted"]
    assert s32["emitted"] == E
    assert np.mean(n32 == n64) >= 0.97
    assert abs(float(t32.sum()) - t64.sum()) <= 1e-6 * E
    assert abs(s32["escaped"] - s64["escaped"]) <= 1e-6 * E
    assert np.abs(t32 - t64).sum() <= 3e-4 * t64.sum()
