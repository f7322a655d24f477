"""Pins of the CPU oracle against what the mathematics and the physics fix
(no GPU).  Each test is chosen so that a plausible slip in the oracle (a
dropped term, a wrong sign, a transposed operand, a wrong constant) fails it.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(cl):
    return oracle.Grid(cl.nx, cl.ny, cl.nz, cl.level_start, cl.rho, cl.child, cl.parent)


def _ulp_err(approx, exact):
    approx = np.asarray(approx, np.float64)
    exact = np.asarray(exact, np.float64)
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    return np.abs(approx - exact) / ulp


# ----------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_u01_open_interval_and_grid():
    xs = [0, 1, 255, 256, 0x7FFFFFFF, 0x80000000, 0xFFFFFF00, 0xFFFFFFFF]
    us = [oracle.u01(x) for x in xs]
    assert min(us) == 2.0 ** -24 and max(us) == 1.0 - 2.0 ** -24
    for x, u in zip(xs, us):
        assert 0.0 < u < 1.0
        k = u * 2.0 ** 24
        assert k == int(k) and int(k) % 2 == 1 and int(k) == ((x >> 8) | 1)


# ----------------------------------------------------------------------------
# elementary functions of the FP32 contract
# ----------------------------------------------------------------------------
def test_one_minus_exp_within_2ulp_of_fp64():
    rng = np.random.default_rng(1)
    tau = np.concatenate([np.geomspace(1e-30, 0.5, 100_000), rng.uniform(0.4, 0.6, 50_000),
                          rng.uniform(0, 80, 100_000)]).astype(np.float32)
    q = oracle.one_minus_exp(tau)
    err = _ulp_err(q, -np.expm1(-tau.astype(np.float64)))
    assert err.max() <= 2.0, err.max()
    assert oracle.one_minus_exp(np.float32([0.0, -1.0, np.nan])).tolist() == [0.0, 0.0, 0.0]
    # around every reduction boundary (k changes at tau = (j + 1/2) ln 2) and far out
    j = np.arange(0, 126)
    edge = ((j + 0.5) * math.log(2))[:, None] * (1.0 + np.linspace(-1e-5, 1e-5, 41))[None, :]
    tau2 = np.concatenate([edge.ravel(), [86.9, 87.0, 87.5, 100.0, 1e30]]).astype(np.float32)
    q2 = oracle.one_minus_exp(tau2)
    assert _ulp_err(q2, -np.expm1(-tau2.astype(np.float64))).max() <= 2.0
    assert np.all(np.diff(q2[:edge.size].reshape(edge.shape), axis=1) >= 0)    # monotone across each boundary


def test_log_within_2ulp_of_fp64():
    rng = np.random.default_rng(2)
    k = rng.integers(0, 1 << 24, 400_000)
    u = (((k >> 0) | 1) * 2.0 ** -24).astype(np.float32)
    u = np.concatenate([u, np.float32([2.0 ** -24, 0.5, 1 - 2.0 ** -24, 0.70710677, 0.7071068])])
    y = oracle.log(u)
    err = _ulp_err(y, np.log(u.astype(np.float64)))
    assert err.max() <= 2.0, err.max()


# ----------------------------------------------------------------------------
# pencil beams: exp(-tau) attenuation and geometry
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("refined", [False, True])
def test_pencil_beam_column_exp_minus_tau(refined):
    n, kabs = 24, 0.37
    cl = I.regular(np.ones((n, 1, 1), np.float32))
    if refined:                       # refine every 3rd cell: same medium, deeper tree
        cl = I.refine_cells(cl, np.arange(0, n, 3))
    G = _grid(cl)
    tally, st, steps = oracle.trace_pencil(G, [0.5, 0.5, 0.0], [0.0, 0.0, 1.0], kabs=kabs)
    assert tally.sum() + st["escaped"] == st["emitted"] == oracle.W_UNIT
    T = st["escaped"] / oracle.W_UNIT
    assert abs(T / math.exp(-kabs * n) - 1.0) < n * 4e-7
    # every root cell (with its children) absorbs W_in (1 - e^-kabs)
    per_root = np.zeros(n)
    owner = np.arange(cl.n_cells)
    for k, p in enumerate(cl.parent):
        owner[cl.n_root + 8 * k: cl.n_root + 8 * k + 8] = p
    np.add.at(per_root, owner, tally)
    expect = np.exp(-kabs * np.arange(n)) * (1 - math.exp(-kabs)) * oracle.W_UNIT
    np.testing.assert_allclose(per_root, expect, rtol=5e-6 * n)
    assert steps == (n if not refined else n + (n // 3) * 1)


def test_pencil_beam_oblique_path_length():
    n, kabs = 16, 0.05
    cl = I.regular(np.ones((n, n, n), np.float32))
    d = np.array([0.3, 0.5, 0.81], np.float64)
    d /= np.linalg.norm(d)
    d32 = d.astype(np.float32)
    tally, st, _ = oracle.trace_pencil(_grid(cl), [0.0, 0.0, 0.0], d32, kabs=kabs)
    L = n / np.abs(d32.astype(np.float64)).max()       # first face of the box hit
    assert abs(st["escaped"] / oracle.W_UNIT / math.exp(-kabs * L) - 1) < 2e-5


def test_unscattered_fraction_is_exp_minus_tau_sca():
    """Pencil beams up a column with albedo 0.5: a package that never scatters
    leaves through the top with one exact weight; the fraction of such
    packages is exp(-tau_sca) (free paths drawn in scattering optical depth)."""
    n, ksca, kabs = 8, 0.125, 0.125                       # tau_sca = tau_abs = 1
    cl = I.regular(np.ones((n, 9, 9), np.float32))
    G = _grid(cl)
    straight, _, _ = oracle.trace_pencil(G, [4.5, 4.5, 0.0], [0.0, 0.0, 1.0], kabs=kabs)
    w_straight = oracle.W_UNIT - int(straight.sum())
    M = 6000
    hits = 0
    for pid in range(M):
        t, st, _ = oracle.trace_pencil(G, [4.5, 4.5, 0.0], [0.0, 0.0, 1.0], kabs=kabs, ksca=ksca, g=0.3,
                                       seed=77, pid=pid)
        hits += st["escaped"] == w_straight
    p = math.exp(-ksca * n)
    assert abs(hits / M - p) < 4 * math.sqrt(p * (1 - p) / M)


def test_zero_density_cells_are_transparent():
    n = 10
    rho = np.zeros((n, 1, 1), np.float32)
    rho[4, 0, 0] = 1.0
    G = _grid(I.regular(rho))
    tally, st, _ = oracle.trace_pencil(G, [0.5, 0.5, 0.0], [0.0, 0.0, 1.0], kabs=0.5, ksca=2.0)
    # only cell 4 can absorb or scatter; cells below it never get a deposit
    assert np.all(tally[:4] == 0)
    assert tally.sum() + st["escaped"] == oracle.W_UNIT


# ----------------------------------------------------------------------------
# conservation (exact, integer) for every source class and grid kind
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("source", [oracle.SRC_BACKGROUND, oracle.SRC_POINT, oracle.SRC_DUST])
@pytest.mark.parametrize("octree", [False, True])
def test_conservation_exact(source, octree):
    if octree:
        w = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0)
    else:
        w = I.config_c2(n=12, n_freq=8)
    cl = w.clouds[0]
    G = _grid(cl)
    f = len(w.dust.nu) - 2
    kw = dict(kabs=w.dust.kabs[f] * cl.ell, ksca=w.dust.ksca[f] * cl.ell, g=0.5, seed=7, freq=f)
    if source == oracle.SRC_POINT:
        pos = np.array([[cl.nx / 2 + 0.3, cl.ny / 3, cl.nz * 0.7]])
        kw.update(ps_pos=pos, ps_cdf=np.float32([1.0]))
    n = 3000
    if source == oracle.SRC_DUST:
        leaf = cl.leaves()
        rng = np.random.default_rng(3)
        dw = rng.integers(0, 2 ** 31, leaf.size).astype(np.uint64)
        dw[::7] = 0
        kw.update(leaf=leaf, dust_w=dw, n_per_cell=2)
        n = 2 * leaf.size
    tally, st, steps = oracle.trace(G, source=source, n_packages=n, want_steps=True, **kw)
    assert int(tally.sum()) + st["escaped"] == st["emitted"]
    assert st["steps"] == int(steps.sum()) and st["capped"] == 0
    assert np.all(tally >= 0)
    if source == oracle.SRC_DUST:
        assert st["emitted"] == 2 * int(dw.sum())
        assert np.all(steps[0::2][dw == 0] == 0)


def test_step_cap_ends_packages_and_conserves():
    cl = I.regular(np.ones((8, 8, 8), np.float32))
    tally, st, steps = oracle.trace(_grid(cl), source=oracle.SRC_BACKGROUND, kabs=0.01, ksca=3.0,
                                    n_packages=500, max_steps=5, want_steps=True)
    assert st["capped"] > 0 and steps.max() == 5
    assert int(tally.sum()) + st["escaped"] == st["emitted"]


def test_same_seed_same_result_other_seed_differs():
    cl = I.regular(np.ones((8, 8, 8), np.float32))
    G = _grid(cl)
    a = oracle.trace(G, source=0, kabs=0.1, ksca=0.2, g=0.3, seed=5, n_packages=2000)[0]
    b = oracle.trace(G, source=0, kabs=0.1, ksca=0.2, g=0.3, seed=5, n_packages=2000)[0]
    c = oracle.trace(G, source=0, kabs=0.1, ksca=0.2, g=0.3, seed=6, n_packages=2000)[0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # packages are independent: two halves add up to the whole
    h1 = oracle.trace(G, source=0, kabs=0.1, ksca=0.2, g=0.3, seed=5, n_packages=1000)[0]
    h2 = oracle.trace(G, source=0, kabs=0.1, ksca=0.2, g=0.3, seed=5, pid_lo=1000, n_packages=1000)[0]
    assert np.array_equal(h1 + h2, a)


# ----------------------------------------------------------------------------
# radiation-field normalisation
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(8, 8, 8), (4, 6, 10)])
def test_background_thin_box_absorbs_4pi_kappa_I(shape):
    """Inside an optically thin box in an isotropic field I, every cell absorbs
    4 pi kabs I per unit rho V (J = I).  Pins the cosine-weighted entry, the
    face choice by area (non-cubic box) and the energy per package (pi I S / N)."""
    nz, ny, nx = shape
    ell, kabs, I_nu = 2.0, 1e-4, 3.0
    cl = I.regular(np.ones(shape, np.float32), ell=ell)
    N = 200_000
    tally, st, _ = oracle.trace(_grid(cl), source=0, kabs=kabs * ell, ksca=0.0, seed=11, n_packages=N)
    e = P.background_package_energy([I_nu], nx, ny, nz, ell, N)
    A = P.absorbed_power(tally[None, :], e, [1.0], cl.rho, P.cell_volumes(_grid(cl), ell))
    ratio = A / (4 * np.pi * kabs * I_nu)
    assert abs(ratio.mean() - 1) < 4e-3
    assert np.all(np.abs(ratio - 1) < 0.12)
    # mean chord of cosine-weighted entry is 4V/S (Cauchy): steps ~ N * n * 2/3 * ...
    assert abs(st["emitted"] - N * oracle.W_UNIT) == 0


def test_point_source_inverse_square():
    """Optically thin cube with a central point source: absorbed power per
    cell = kabs rho L <1/(4 pi r^2)>_cell, i.e. J = L / (16 pi^2 r^2)."""
    n, kabs, L = 24, 1e-4, 5.0
    cl = I.regular(np.ones((n, n, n), np.float32))
    N = 400_000
    c = n / 2
    tally, st, _ = oracle.trace(_grid(cl), source=1, kabs=kabs, ksca=0.0, seed=3, n_packages=N,
                                ps_pos=np.array([[c, c, c]]), ps_cdf=np.float32([1.0]))
    absorbed = tally * (L / N / oracle.W_UNIT)
    # exact cell average of 1/(4 pi r^2) by a 6^3 midpoint rule
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    sub = (np.arange(6) + 0.5) / 6
    inv = np.zeros((n, n, n))
    for a in sub:
        for b in sub:
            for cc in sub:
                r2 = (i + a - c) ** 2 + (j + b - c) ** 2 + (k + cc - c) ** 2
                inv += 1.0 / (4 * np.pi * r2)
    inv /= 216
    expect = (kabs * L * inv).ravel()
    r = np.sqrt((i + 0.5 - c) ** 2 + (j + 0.5 - c) ** 2 + (k + 0.5 - c) ** 2).ravel()
    far = r >= 4
    ratio = absorbed[far].sum() / expect[far].sum()
    assert abs(ratio - 1) < 5e-3
    # slope of the shell averages in log J vs log r is -2
    bins = np.arange(4, 11)
    mids, vals = [], []
    for lo, hi in zip(bins[:-1], bins[1:]):
        m = (r >= lo) & (r < hi)
        mids.append(np.mean(r[m]))
        vals.append(absorbed[m].mean())
    slope = np.polyfit(np.log(mids), np.log(vals), 1)[0]
    assert abs(slope + 2) < 0.05
    # isotropy: the six half-spaces around the source absorb equal shares
    a3 = absorbed.reshape(n, n, n)
    h = n // 2
    halves = [a3[:h].sum(), a3[h:].sum(), a3[:, :h].sum(), a3[:, h:].sum(), a3[:, :, :h].sum(), a3[:, :, h:].sum()]
    tot = a3.sum()
    assert max(abs(x / tot - 0.5) for x in halves) < 0.01


def _cube_transmission_quadrature(tau_side, n=96):
    """Escape probability of cosine-weighted rays entering a unit cube through
    one face with absorption coefficient tau_side (deterministic midpoint
    quadrature over entry point (x, y), mu^2 and azimuth)."""
    g = (np.arange(n) + 0.5) / n
    x, y = np.meshgrid(g, g, indexing="ij")
    tot = 0.0
    for m2 in g:
        mu = math.sqrt(m2)
        st = math.sqrt(1 - m2)
        for ph in 2 * np.pi * g:
            dx, dy = st * math.cos(ph), st * math.sin(ph)
            tz = 1.0 / mu
            tx = np.where(dx > 0, (1 - x) / dx, np.where(dx < 0, -x / dx, np.inf)) if dx != 0 else np.inf
            ty = np.where(dy > 0, (1 - y) / dy, np.where(dy < 0, -y / dy, np.inf)) if dy != 0 else np.inf
            Lp = np.minimum(np.minimum(tx, ty), tz)
            tot += np.exp(-tau_side * Lp).mean()
    return tot / (n * n)


@pytest.mark.parametrize("layout", ["1cube", "2cube", "2cube_refined"])
def test_brute_force_escape_probability_small_grids(layout):
    """Albedo 0: the escaped fraction of background packages equals the
    quadrature of exp(-tau(path)) over cosine-weighted entry (same for every
    face by symmetry)."""
    tau_side = 1.3
    if layout == "1cube":
        cl = I.regular(np.ones((1, 1, 1), np.float32)); k = tau_side
    else:
        cl = I.regular(np.ones((2, 2, 2), np.float32)); k = tau_side / 2
        if layout == "2cube_refined":
            cl = I.refine_cells(cl, [0, 3, 6])
            cl = I.refine_cells(cl, [cl.level_start[1] + 1, cl.level_start[1] + 9])
    N = 400_000
    tally, st, _ = oracle.trace(_grid(cl), source=0, kabs=k, ksca=0.0, seed=21, n_packages=N)
    p_mc = st["escaped"] / (N * oracle.W_UNIT)
    p_q = _cube_transmission_quadrature(tau_side)
    assert abs(p_mc - p_q) < 2.5e-3, (p_mc, p_q)


def test_octree_refinement_does_not_change_root_absorption():
    """A uniform cloud refined arbitrarily is the same medium: with the same
    random numbers the absorption summed per root cell matches the unrefined
    run up to rounding-level path differences."""
    n = 6
    base = I.regular(np.ones((n, n, n), np.float32) * 2.0)
    rng = np.random.default_rng(4)
    ref = I.refine_cells(base, rng.choice(base.n_cells, 60, replace=False))
    lv2 = np.arange(ref.level_start[1], ref.level_start[2])
    ref = I.refine_cells(ref, rng.choice(lv2, 100, replace=False))
    kw = dict(source=0, kabs=0.08, ksca=0.15, g=0.4, seed=9, n_packages=30_000)
    t0, s0, _ = oracle.trace(_grid(base), **kw)
    t1, s1, _ = oracle.trace(_grid(ref), **kw)
    # map every cell to its root ancestor
    owner = np.arange(ref.n_cells)
    par_of_cell = np.full(ref.n_cells, -1)
    for k, p in enumerate(ref.parent):
        par_of_cell[ref.n_root + 8 * k: ref.n_root + 8 * k + 8] = p
    for _ in range(ref.n_levels):
        owner = np.where(owner >= ref.n_root, par_of_cell[owner], owner)
    per_root = np.bincount(owner, weights=t1.astype(np.float64), minlength=ref.n_root)
    rel = np.abs(per_root - t0.astype(np.float64)) / t0.sum()
    assert rel.max() < 2e-3
    assert abs(s1["escaped"] - s0["escaped"]) / s0["emitted"] < 2e-3
    assert s1["steps"] > s0["steps"]


def test_point_sources_chosen_in_proportion_to_luminosity():
    """Several point sources (Sect. 3.1 tests one; the reading: a package
    picks its source with probability L_k / sum L at its frequency, all
    packages carrying equal energy).  An opaque cube keeps each package's
    energy in its source's cell: the cells' shares are the luminosity
    fractions."""
    cl = I.regular(np.ones((5, 5, 5), np.float32))
    L = np.array([[3.0], [1.0], [4.0]])
    pos = np.array([[0.5, 0.5, 0.5], [2.5, 2.5, 2.5], [4.5, 3.5, 0.5]])
    cdf = P.point_source_cdf(L)[0]
    N = 60_000
    t, st, _ = oracle.trace(_grid(cl), source=1, kabs=200.0, ksca=0.0, seed=4, n_packages=N,
                            ps_pos=pos, ps_cdf=cdf)
    cells = [int(p[0]) + 5 * (int(p[1]) + 5 * int(p[2])) for p in pos]
    share = t[cells] / st["emitted"]
    expect = L[:, 0] / L.sum()
    assert np.all(np.abs(share - expect) < 4 * np.sqrt(expect * (1 - expect) / N) + 1e-3), (share, expect)


# ----------------------------------------------------------------------------
# scattering
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("g", [0.0, 0.5])
def test_mean_square_absorption_distance_point_source(g):
    """Point source in a (practically) infinite uniform medium, absorption as
    continuous attenuation, Poisson scattering with mean cosine g: the
    direction autocorrelation along the path is exp(-ks (1-g) l), so the
    energy-weighted mean square distance of absorption from the source is
    exactly 2 / (ka (ka + ks (1 - g))).  Pins the free-path draws after every
    scattering and the transport effect of the phase function."""
    n, ka, ks = 96, 0.1, 0.3
    cl = I.regular(np.ones((n, n, n), np.float32))
    c = n / 2
    N = 20_000
    tally, st, _ = oracle.trace(_grid(cl), source=1, kabs=ka, ksca=ks, g=g, seed=13, n_packages=N,
                                ps_pos=np.array([[c, c, c]]), ps_cdf=np.float32([1.0]))
    assert st["escaped"] < 1e-3 * st["emitted"]
    idx = np.nonzero(tally)[0]
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    r2 = (i + 0.5 - c) ** 2 + (j + 0.5 - c) ** 2 + (k + 0.5 - c) ** 2 + 0.25   # cell average of r^2
    m = np.sum(tally[idx] * r2) / tally[idx].sum()
    expect = 2.0 / (ka * (ka + ks * (1 - g)))
    assert abs(m / expect - 1) < 0.04, (m, expect)

@pytest.mark.parametrize("g", [0.0, 0.5, -0.3, 0.9])
def test_hg_moments(g):
    n = 200_000
    d0 = np.array([0.3, -0.4, np.sqrt(1 - 0.25)], np.float32)
    cosv, dout = oracle.hg_samples(g, d0, 123, n)
    se = 1.0 / math.sqrt(n)
    assert abs(cosv.mean() - g) < 4 * se
    assert abs((cosv.astype(np.float64) ** 2).mean() - (1 + 2 * g * g) / 3) < 4 * se
    np.testing.assert_allclose(np.linalg.norm(dout.astype(np.float64), axis=1), 1.0, atol=3e-7)
    # azimuthal symmetry about d0: the perpendicular part averages to zero
    perp = dout - cosv[:, None] * d0[None, :]
    assert np.abs(perp.mean(axis=0)).max() < 4 * se


def test_hg_along_z_branch():
    d0 = np.array([0.0, 0.0, -1.0], np.float32)
    cosv, _ = oracle.hg_samples(0.6, d0, 5, 100_000)
    assert abs(cosv.mean() - 0.6) < 4 / math.sqrt(100_000)


# ----------------------------------------------------------------------------
# noise law (paper Sect. 3.1: noise ~ N^-1/2)
# ----------------------------------------------------------------------------
def test_noise_scales_as_inverse_sqrt_n():
    cl = I.regular(np.ones((6, 6, 6), np.float32))
    G = _grid(cl)

    def rms(N):
        a = oracle.trace(G, source=0, kabs=0.1, ksca=0.1, seed=100, n_packages=N)[0] / N
        b = oracle.trace(G, source=0, kabs=0.1, ksca=0.1, seed=200, n_packages=N)[0] / N
        return np.sqrt(np.mean((a - b) ** 2))

    r = rms(4000) / rms(64000)
    assert 3.3 < r < 4.8       # sqrt(16) = 4


def test_noise_grows_as_2_to_the_level_for_background_heating():
    """Sect. 3.1: each level of refinement cuts the packages crossing a cell
    by four, so the relative noise of a cell's absorbed power grows as 2^L
    for background heating.  Thin uniform box, root cells split once and
    some of those split again: the scatter of absorbed power per volume
    among the leaves of one level doubles from level to level."""
    cl = I.regular(np.ones((4, 4, 4), np.float32))
    cl = I.refine_cells(cl, np.arange(32, 64))                       # upper half: level 1
    l1 = np.arange(cl.level_start[1], cl.level_start[2])
    cl = I.refine_cells(cl, l1[::2])                                 # half of those: level 2
    G = _grid(cl)
    t, st, _ = oracle.trace(G, source=0, kabs=1e-3, ksca=0.0, seed=31, n_packages=400_000)
    vol = 8.0 ** -np.repeat(np.arange(3), np.diff(cl.level_start))
    leaf = cl.child < 0
    a = t / vol
    rel = []
    for L in range(3):
        m = leaf & (np.repeat(np.arange(3), np.diff(cl.level_start)) == L)
        rel.append(a[m].std() / a[m].mean())
    assert 1.5 < rel[1] / rel[0] < 2.7 and 1.5 < rel[2] / rel[1] < 2.7, rel


# ----------------------------------------------------------------------------
# FP64 physics
# ----------------------------------------------------------------------------
def test_planck_integrates_to_stefan_boltzmann():
    sigma = 5.670374419e-5          # CODATA 2018
    for T in (10.0, 300.0, 6000.0):
        nu = np.geomspace(1e8, 1e17, 200_001)
        I_ = np.sum(P.trapezoid_weights(nu) * P.planck_nu(nu, T))
        assert abs(I_ / (sigma * T ** 4 / np.pi) - 1) < 1e-6


def test_planck_derivative():
    nu = np.geomspace(1e11, 1e15, 50)
    for T in (5.0, 50.0, 900.0):
        h = T * 1e-6
        fd = (P.planck_nu(nu, T + h) - P.planck_nu(nu, T - h)) / (2 * h)
        ok = P.H_PLANCK * nu / (P.K_BOLTZ * T) < 300.0
        np.testing.assert_allclose(P.dplanck_dT(nu, T)[ok], fd[ok], rtol=1e-6)


def test_trapezoid_weights_exact_for_linear():
    nu = np.geomspace(3e11, 3e15, 64)
    w = P.trapezoid_weights(nu)
    assert abs(w.sum() / (nu[-1] - nu[0]) - 1) < 1e-14
    assert abs(np.sum(w * nu) / (0.5 * (nu[-1] ** 2 - nu[0] ** 2)) - 1) < 1e-13


@pytest.mark.parametrize("beta", [1.0, 2.0])
@pytest.mark.parametrize("W", [1.0, 1e-3, 1e-8])
def test_temperature_closed_form_diluted_blackbody(beta, W):
    """Optically thin dust in a field W B(T*) with kappa ~ nu^beta is at
    T = W^(1/(4+beta)) T* (infinite frequency range)."""
    Tstar = 200.0
    nu = np.geomspace(1e9, 1e16, 6000)
    kabs = (nu / 1e12) ** beta
    A = 4 * np.pi * np.sum(P.trapezoid_weights(nu) * kabs * W * P.planck_nu(nu, Tstar))
    T = P.temperature(A, nu, kabs)
    assert abs(T / (W ** (1 / (4 + beta)) * Tstar) - 1) < 1e-4


def test_temperature_blackbody_field_on_coarse_grid_and_limits():
    nu = I.frequency_grid(64)
    kabs = (nu / 1e14) ** 2
    for Tstar in (15.0, 120.0, 1500.0):
        A = P.emission_integral(Tstar, nu, kabs)      # W = 1: T = T* for any quadrature
        assert abs(P.temperature(A, nu, kabs) / Tstar - 1) < 1e-10
    assert P.temperature(0.0, nu, kabs) == P.T_MIN
    assert P.temperature(1e300, nu, kabs) == P.T_MAX


def test_thin_cube_mc_temperature_matches_closed_form():
    """End to end in FP64 after the FP32 tracer: a thin cube in W B(T*) reaches
    the temperature of the same quadrature's equilibrium."""
    nu = I.frequency_grid(16)
    kabs = 1e-6 * (nu / 1e14) ** 2
    W, Tstar = 1e-6, 3000.0
    I_nu = W * P.planck_nu(nu, Tstar)
    n, ell, N = 6, 1.0, 60_000
    cl = I.regular(np.ones((n, n, n), np.float32), ell=ell)
    G = _grid(cl)
    tal = np.zeros((len(nu), cl.n_cells), np.int64)
    for f in range(len(nu)):
        tal[f] = oracle.trace(G, source=0, kabs=kabs[f] * ell, ksca=0.0, seed=1, freq=f,
                              n_packages=N)[0]
    e = P.background_package_energy(I_nu, n, n, n, ell, N)
    A = P.absorbed_power(tal, e, nu, cl.rho, cl.volumes())
    T = P.temperatures(A, nu, kabs)
    A_exact = 4 * np.pi * np.sum(P.trapezoid_weights(nu) * kabs * I_nu)
    T_exact = P.temperature(A_exact, nu, kabs)
    assert abs(T.mean() / T_exact - 1) < 2e-3
    assert np.all(np.abs(T / T_exact - 1) < 0.02)


def test_dust_weights():
    L = np.array([0.0, 1.0, 2.5, 5.0, 5.0 * (1 - 2 ** -40)])
    W, e = P.dust_weights(L, 3)
    assert W[3] == 2 ** 31 and W[0] == 0 and W[1] == round(2 ** 31 / 5)
    assert W[4] == 2 ** 31
    assert abs(e * 2 ** 31 * 3 - 5.0) < 1e-12


def test_faint_dust_package_is_not_dumped_into_its_own_cell():
    """A dust package carries W0 = 2^32 L_c / max L; a faint one (small W0)
    must deposit its energy along the same path as a bright one, scaled by
    W0, instead of ending at once in the emitting cell (which would make the
    cell re-absorb its own emission)."""
    cl = I.regular(np.ones((6, 6, 6), np.float32))
    leaf = cl.leaves()
    G = _grid(cl)
    kw = dict(source=oracle.SRC_DUST, kabs=0.05, ksca=0.0, seed=4, leaf=leaf, n_per_cell=1, n_packages=leaf.size)
    big = oracle.trace(G, dust_w=np.full(leaf.size, 2 ** 31, np.uint64), **kw)[0].astype(np.float64)
    small = oracle.trace(G, dust_w=np.full(leaf.size, 2 ** 11, np.uint64), **kw)[0].astype(np.float64)
    assert small.sum() > 0
    np.testing.assert_allclose(small / small.sum(), big / big.sum(), atol=2e-3)


def test_self_absorption_counter():
    """Deposits a dust package makes before it first leaves its emission cell:
    never more than the cell's total, equal to it in a one-cell grid, and the
    local absorption of an optically thick cell is most of its emission."""
    cl = I.regular(np.ones((6, 6, 6), np.float32))
    leaf = cl.leaves()
    kw = dict(source=oracle.SRC_DUST, ksca=0.3, g=0.2, seed=8, leaf=leaf, n_per_cell=2, n_packages=2 * leaf.size,
              dust_w=np.full(leaf.size, 2 ** 31, np.uint64))
    self_t = np.zeros(cl.n_cells, np.int64)
    tally, st, _ = oracle.trace(_grid(cl), kabs=0.2, self_tally=self_t, **kw)
    assert np.all(self_t <= tally) and self_t.sum() > 0
    one = I.regular(np.ones((1, 1, 1), np.float32))
    s1 = np.zeros(1, np.int64)
    t1, _, _ = oracle.trace(_grid(one), kabs=0.7, self_tally=s1, leaf=one.leaves(), dust_w=np.full(1, 2 ** 31, np.uint64),
                            source=oracle.SRC_DUST, ksca=0.4, g=0.0, seed=3, n_per_cell=500, n_packages=500)
    assert s1[0] == t1[0] > 0
    s2 = np.zeros(cl.n_cells, np.int64)
    t2, st2, _ = oracle.trace(_grid(cl), kabs=20.0, self_tally=s2, **kw)
    assert s2.sum() > 0.85 * st2["emitted"]


def test_ali_update_reaches_the_same_fixed_point():
    """The diagonal-operator update has the plain update's fixed point: with
    A = A_ext + A_self and A_self = beta E(T) at T = T*, both return T*."""
    nu = I.frequency_grid(16)
    kabs = (nu / 1e14) ** 2
    Tstar = 85.0
    E = P.emission_integral(Tstar, nu, kabs)
    for beta in (0.0, 0.3, 0.9):
        A = E
        A_self = beta * E
        assert abs(P.temperature_ali(A, A_self, Tstar, nu, kabs) / Tstar - 1) < 1e-9
    # away from the fixed point ALI moves further toward it than the plain update
    T_old, beta, A_ext = 40.0, 0.8, 0.2 * E
    A_self = beta * P.emission_integral(T_old, nu, kabs)
    plain = P.temperature(A_ext + A_self, nu, kabs)
    ali = P.temperature_ali(A_ext + A_self, A_self, T_old, nu, kabs)
    assert plain < ali <= Tstar * 1.0001


def test_weighted_dust_sampling_allocation():
    """Packages follow the luminosity, the cap holds, every emitting cell
    gets a package, and packages x weight x unit energy return each cell's
    luminosity (to rounding)."""
    rng = np.random.default_rng(5)
    L = np.exp(rng.normal(0, 3, 2000))
    L[7] = L.max() * 50                       # one very bright cell
    L[::13] = 0.0
    u, e_uni = P.dust_weights(L, 1)
    N, cap = 20000, 300
    n, pref, W, e = P.weighted_dust_sampling(u, e_uni, N, cap)
    assert n.max() <= cap and n[7] == cap
    assert np.all((n > 0) == (u > 0)) and pref[-1] == n.sum()
    assert np.all(W <= 2 ** 31) and W.max() == 2 ** 31
    emitted = n.astype(np.float64) * W.astype(np.float64) * e
    ok = u > 2 ** 12
    np.testing.assert_allclose(emitted[ok], L[ok], rtol=2e-3)
    # away from the cap and from the one-package floor, n follows L
    mid = (n > 5) & (n < cap)
    ratio = n[mid] / (N * L[mid] / L.sum())
    assert np.all((ratio > 0.8) & (ratio < 1.3))


def test_weighted_dust_tracing_conserves_and_uses_prefix():
    cl = I.regular(np.ones((5, 5, 5), np.float32))
    leaf = cl.leaves()
    rng = np.random.default_rng(6)
    u = rng.integers(0, 2 ** 31, leaf.size).astype(np.uint64)
    n, pref, W, e = P.weighted_dust_sampling(u, 1.0, 3 * leaf.size, 40)
    tally, st, steps = oracle.trace(_grid(cl), source=oracle.SRC_DUST, kabs=0.3, ksca=0.2, g=0.1, seed=2, leaf=leaf,
                                    dust_w=W, dust_prefix=pref, n_packages=int(pref[-1]), want_steps=True)
    assert int(tally.sum()) + st["escaped"] == st["emitted"] == int((n * W).sum())


def test_weighted_reweight_keeps_counts_and_energy():
    rng = np.random.default_rng(12)
    L0 = np.exp(rng.normal(0, 2, 500))
    u0, e0 = P.dust_weights(L0, 1)
    n, pref, W0, e_0 = P.weighted_dust_sampling(u0, e0, 3000, 40)
    L1 = L0 * np.exp(rng.normal(0, 0.3, 500))          # new temperatures
    u1, e1 = P.dust_weights(L1, 1)
    W1, e_1 = P.weighted_dust_reweight(u1, e1, pref)
    assert W1.max() == 2 ** 31 and np.all((W1 > 0) <= (n > 0))
    ok = (n > 0) & (u1 > 2 ** 16)
    np.testing.assert_allclose(n[ok] * W1[ok].astype(np.float64) * e_1, L1[ok], rtol=1e-4)


def test_package_schedule_and_reference_weights():
    n = P.package_schedule(1000, 200000, 5)
    assert n[0] == 1000 and n[-1] == 200000
    r = n[1:].astype(np.float64) / n[:-1]
    np.testing.assert_allclose(r, 200.0 ** 0.25, rtol=1e-3)        # log n linear in k
    w = P.reference_weights([4, 4, 4, 4])
    np.testing.assert_allclose(w, [1, 1 / 2, 1 / 3, 1 / 4])
    assert P.package_schedule(7, 9, 1)[0] == 9


def test_reference_field_running_mean_and_special_cases():
    """The reference emission is the package-weighted mean of the emissions
    seen so far; a first iteration (L_ref = 0) is plain emission-weighted
    sampling of L; no change gives no packages."""
    rng = np.random.default_rng(13)
    Ls = [np.exp(rng.normal(0, 1, 300)) for _ in range(4)]
    n = np.array([100, 400, 1600, 6400])
    w = P.reference_weights(n)
    L_ref = np.zeros(300)
    for k in range(4):
        u, neg, e, L_ref = P.reference_delta(Ls[k], L_ref, w[k])
    np.testing.assert_allclose(L_ref, sum(nk * L for nk, L in zip(n, Ls)) / n.sum(), rtol=1e-13)
    # first iteration: the same weights as the uniform dust weights of L
    u1, neg1, e1, _ = P.reference_delta(Ls[0], np.zeros(300), 1.0)
    u0, e0 = P.dust_weights(Ls[0], 1)
    np.testing.assert_array_equal(u1, u0)
    assert not neg1.any() and e1 == e0
    # a converged emission traces nothing
    u2, neg2, e2, L2 = P.reference_delta(Ls[1], Ls[1], 0.5)
    assert e2 == 0.0 and not u2.any() and np.array_equal(L2, Ls[1])
    # signs and magnitudes: units x e_uni return |d|
    u3, neg3, e3, _ = P.reference_delta(Ls[2], Ls[3], 0.3)
    d = Ls[2] - Ls[3]
    np.testing.assert_array_equal(neg3, d < 0)
    np.testing.assert_allclose(u3 * e3, np.abs(d), rtol=1e-9, atol=e3)
    Wp, Wn = P.split_allocation(u3, neg3)
    np.testing.assert_array_equal(Wp + Wn, u3)
    assert not Wp[neg3].any() and not Wn[~neg3].any()


def test_reference_field_correction_is_unbiased_by_linearity():
    """Tracing the change d = L_b - L_a (both signs, weighted sampling) and
    adding it to the absorption of L_a gives, in the mean over seeds, the
    absorption of L_b (the estimator the reference field relies on)."""
    cl = I.regular(np.full((4, 4, 4), 2.0, np.float32))
    leaf = cl.leaves()
    G = _grid(cl)
    rng = np.random.default_rng(17)
    L_a = np.exp(rng.normal(0, 1, leaf.size))
    L_b = L_a * np.exp(rng.normal(0, 0.5, leaf.size))

    def absorbed(W, e, seed, n_pk, **kw):
        t = oracle.trace(G, source=oracle.SRC_DUST, kabs=0.25, ksca=0.0, g=0.0, seed=seed, leaf=leaf, dust_w=W,
                         n_packages=n_pk, **kw)[0]
        return t.astype(np.float64) * e

    nl = leaf.size
    u_b, e_b = P.dust_weights(L_b, 64)          # direct: 64 packages per cell
    A_b = np.mean([absorbed(u_b, e_b, s, 64 * nl, n_per_cell=64) for s in (1, 2)], axis=0)
    u_a, e_a = P.dust_weights(L_a, 64)
    A_a = np.mean([absorbed(u_a, e_a, s, 64 * nl, n_per_cell=64) for s in (3, 4)], axis=0)
    u, neg, e_uni, _ = P.reference_delta(L_b, L_a, 1.0)
    n, pref, W, e_w = P.weighted_dust_sampling(u, e_uni, 64 * nl, 10 ** 6)
    Wp, Wn = P.split_allocation(W, neg)
    n_pk = int(pref[-1])
    dA = np.mean([absorbed(Wp, e_w, s, n_pk, dust_prefix=pref) - absorbed(Wn, e_w, s, n_pk, dust_prefix=pref)
                  for s in (5, 6)], axis=0)
    tot_b, tot_ref = A_b.sum(), (A_a + dA).sum()
    assert abs(tot_ref / tot_b - 1) < 0.02, (tot_ref, tot_b)


def test_reference_mean_noise_falls_with_iterations():
    """Mean reading at fixed emission: the running package-weighted mean of
    independent absorption estimates has a seed-to-seed scatter that falls
    as (number of iterations)^-1/2 (Sect. 2.1.2's ideal case)."""
    cl = I.regular(np.full((4, 4, 4), 1.0, np.float32))
    leaf = cl.leaves()
    G = _grid(cl)
    L = np.exp(np.random.default_rng(23).normal(0, 1, leaf.size))
    u, e = P.dust_weights(L, 4)

    def run(seed, K):
        n = P.package_schedule(4 * leaf.size, 4 * leaf.size, K)
        wk = P.reference_weights(n)
        A = np.zeros(leaf.size)
        for k in range(K):
            t = oracle.trace(G, source=oracle.SRC_DUST, kabs=0.3, ksca=0.0, g=0.0, seed=seed, iteration=k + 1,
                             leaf=leaf, dust_w=u, n_per_cell=4, n_packages=4 * leaf.size)[0]
            A = P.reference_update(A, t[leaf] * e, wk[k])
        return A

    def scatter(K):
        a, b = run(1, K), run(2, K)
        return float(np.sqrt(np.mean(((a - b) / (0.5 * (a + b))) ** 2)))

    s1, s4 = scatter(1), scatter(4)
    assert 0.35 < s4 / s1 < 0.65, (s1, s4)          # 1/sqrt(4) = 0.5
