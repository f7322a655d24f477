"""Seeded synthetic inputs: clouds, octrees, frequency grids, dust and source
tables.

This module holds no step of the transport method; it only builds the inputs
that both the CUDA path and the CPU oracle consume (the paper's own inputs --
an MHD snapshot, the Mathis 1983 field and the DustEM dust model, Sect. 2.2 --
are replaced by lognormal Gaussian-random-field clouds, diluted blackbodies and
a power-law opacity).  It imports nothing from the CUDA binding.

Grid layout (Sect. 2.1.1): the cell vector starts with the root grid in
x-fastest order (c = i + nx (j + ny k)), followed by all cells of hierarchy
level 2, then level 3, and so on.  Each octet is contiguous, its cells ordered
by octant o = ox + 2 oy + 4 oz, and octets of a level follow the order of
their parents.  ``child[c]`` is the index of the first cell of c's octet or
-1 for a leaf; ``parent[k]`` is the parent of octet k (cells n_root + 8k ..
n_root + 8k + 7).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PC_CM = 3.0856775814913673e18
C_LIGHT = 2.99792458e10
NU_1UM = C_LIGHT / 1e-4               # frequency of 1 micron (Hz)
# blackbody constants used to build input spectra (cgs)
_H = 6.62607015e-27
_K = 1.380649e-16
_SIGMA_SB = 5.670374419e-5


@dataclass
class Cloud:
    nx: int
    ny: int
    nz: int
    level_start: np.ndarray           # int64 [n_levels + 1]
    rho: np.ndarray                   # float32 [n_cells] (parents hold their mean; unused)
    child: np.ndarray                 # int32 [n_cells]
    parent: np.ndarray                # int32 [n_octets]
    ell: float = 1.0                  # root-cell side (cm)

    @property
    def n_root(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_cells(self) -> int:
        return int(self.rho.size)

    @property
    def n_levels(self) -> int:
        return int(self.level_start.size - 1)

    def leaves(self) -> np.ndarray:
        return np.nonzero(self.child < 0)[0].astype(np.int32)

    def level_of(self) -> np.ndarray:
        lv = np.zeros(self.n_cells, np.int32)
        for L in range(self.n_levels):
            lv[self.level_start[L]:self.level_start[L + 1]] = L
        return lv

    def volumes(self) -> np.ndarray:
        return (self.ell * np.ldexp(1.0, -self.level_of())) ** 3

    def paper_encoding(self) -> np.ndarray:
        """Density vector with the paper's link encoding: a refined cell holds
        minus the index of its first child (exact while indices < 2^24)."""
        v = self.rho.astype(np.float32).copy()
        par = self.child >= 0
        v[par] = -self.child[par].astype(np.float32)
        return v

    def cells_per_level(self) -> np.ndarray:
        return np.diff(self.level_start).astype(np.int64)


def regular(rho3d, ell: float = 1.0) -> Cloud:
    """One-level cloud from a (nz, ny, nx) density array."""
    rho3d = np.asarray(rho3d, np.float32)
    nz, ny, nx = rho3d.shape
    n = nx * ny * nz
    return Cloud(nx, ny, nz, np.array([0, n], np.int64), rho3d.ravel().copy(),
                 np.full(n, -1, np.int32), np.zeros(0, np.int32), ell)


def _block_mean(a, f):
    nz, ny, nx = a.shape
    return a.reshape(nz // f, f, ny // f, f, nx // f, f).mean(axis=(1, 3, 5))


def _block_max(a, f):
    nz, ny, nx = a.shape
    return a.reshape(nz // f, f, ny // f, f, nx // f, f).max(axis=(1, 3, 5))


def octree_from_fine(fine, root_n: int, max_refine: int, threshold: float, ell: float = 1.0,
                     mean=None, rule: str = "max") -> Cloud:
    """Octree on a root grid of root_n^3 cells from a fine cube of side
    root_n 2^max_refine: a cell is refined while the density inside it
    exceeds ``threshold`` times the global mean -- anywhere in the cell on the
    fine grid (rule "max") or on average over the cell (rule "mean") -- down
    to max_refine levels of refinement.  Every cell holds its block mean."""
    fine = np.asarray(fine, np.float64)
    N = fine.shape[0]
    assert fine.shape == (N, N, N) and N == root_n << max_refine
    assert rule in ("max", "mean")
    gmean = float(fine.mean()) if mean is None else float(mean)
    means = [_block_mean(fine, 1 << (max_refine - L)) if L < max_refine else fine
             for L in range(max_refine + 1)]
    crit = means if rule == "mean" else [_block_max(fine, 1 << (max_refine - L)) if L < max_refine else fine
                                         for L in range(max_refine + 1)]
    # level 0: root cells in x-fastest order
    k, j, i = np.meshgrid(np.arange(root_n), np.arange(root_n), np.arange(root_n), indexing="ij")
    coords = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)      # (n, 3) as (i, j, k)
    rho_parts, child_parts, parent_parts, starts = [], [], [], [0]
    offset = 0
    for L in range(max_refine + 1):
        m = means[L][coords[:, 2], coords[:, 1], coords[:, 0]]
        n_L = coords.shape[0]
        refine = ((crit[L][coords[:, 2], coords[:, 1], coords[:, 0]] > threshold * gmean) if L < max_refine
                  else np.zeros(n_L, bool))
        child = np.full(n_L, -1, np.int32)
        nref = int(refine.sum())
        next_start = offset + n_L
        child[refine] = next_start + 8 * np.arange(nref, dtype=np.int64)
        rho_parts.append(m.astype(np.float32))
        child_parts.append(child)
        if nref:
            parents_global = offset + np.nonzero(refine)[0]
            parent_parts.append(parents_global.astype(np.int32))
            pc = coords[refine]
            o = np.arange(8)
            off = np.stack([o & 1, (o >> 1) & 1, (o >> 2) & 1], axis=1)
            coords = (2 * pc[:, None, :] + off[None, :, :]).reshape(-1, 3)
        offset = next_start
        starts.append(offset)
        if nref == 0:
            break
    rho = np.concatenate(rho_parts)
    child = np.concatenate(child_parts)
    parent = np.concatenate(parent_parts) if parent_parts else np.zeros(0, np.int32)
    return Cloud(root_n, root_n, root_n, np.array(starts, np.int64), rho, child, parent, ell)


def refine_cells(cloud: Cloud, cells) -> Cloud:
    """Split the given leaves of the LAST level into octets holding the same
    density (for tests: a refined uniform cloud is physically unchanged)."""
    cells = np.sort(np.asarray(cells, np.int64))
    last0, last1 = cloud.level_start[-2], cloud.level_start[-1]
    assert np.all((cells >= last0) & (cells < last1)) and np.all(cloud.child[cells] < 0)
    n = cloud.n_cells
    child = cloud.child.copy()
    child[cells] = n + 8 * np.arange(cells.size)
    rho = np.concatenate([cloud.rho, np.repeat(cloud.rho[cells], 8)])
    child = np.concatenate([child, np.full(8 * cells.size, -1, np.int32)])
    parent = np.concatenate([cloud.parent, cells.astype(np.int32)])
    starts = np.concatenate([cloud.level_start, [n + 8 * cells.size]])
    return Cloud(cloud.nx, cloud.ny, cloud.nz, starts, rho, child, parent, cloud.ell)


def gaussian_random_field(n: int, seed: int, slope: float = -3.5) -> np.ndarray:
    """Periodic Gaussian random field on n^3 with power spectrum P(k) ~ k^slope
    (k = 0 removed), normalised to zero mean and unit variance.  White noise
    from numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    f = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.rfftfreq(n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    g = np.fft.irfftn(f * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_density(n: int, seed: int, sigma: float = 1.5, slope: float = -3.5) -> np.ndarray:
    """rho = exp(sigma g - sigma^2 / 2): lognormal with mean 1."""
    g = gaussian_random_field(n, seed, slope)
    return np.exp(sigma * g - 0.5 * sigma * sigma)


def frequency_grid(n: int = 64, lo: float = 3e11, hi: float = 3e15) -> np.ndarray:
    return np.geomspace(lo, hi, n)


def blackbody(nu, T):
    """Input spectra only: 2 h nu^3 / c^2 / (exp(h nu / k T) - 1)."""
    nu = np.asarray(nu, np.float64)
    with np.errstate(over="ignore"):
        return 2.0 * _H * nu ** 3 / C_LIGHT ** 2 / np.expm1(_H * nu / (_K * T))


def diluted_blackbodies(nu, temps=(3500.0, 6000.0, 25000.0), dilutions=(4e-13, 1e-13, 1e-16)):
    """Background intensity I_nu = sum_k W_k B_nu(T_k) (stand-in for the Mathis field)."""
    return sum(w * blackbody(nu, t) for t, w in zip(temps, dilutions))


def stellar_luminosity(nu, T_star: float, L_bol: float):
    """L_nu of a blackbody star of bolometric luminosity L_bol (erg/s)."""
    return L_bol * np.pi * blackbody(nu, T_star) / (_SIGMA_SB * T_star ** 4)


@dataclass
class Dust:
    nu: np.ndarray
    kabs: np.ndarray                  # cross section per density unit (cm^2)
    ksca: np.ndarray
    g: np.ndarray


def power_law_dust(nu, kext_1um: float, beta: float = 2.0, albedo_max: float = 0.6,
                   nu0: float = 1e14, g: float = 0.5) -> Dust:
    """kappa_ext ~ nu^beta normalised at 1 micron, albedo 0.6 / (1 + (nu0/nu)^2)."""
    nu = np.asarray(nu, np.float64)
    kext = kext_1um * (nu / NU_1UM) ** beta
    alb = albedo_max / (1.0 + (nu0 / nu) ** 2)
    return Dust(nu, (1.0 - alb) * kext, alb * kext, np.full(nu.shape, g))


@dataclass
class Workload:
    name: str
    clouds: list
    dust: Dust
    bg_I: list                        # per cloud: I_nu [n_freq] or None
    ps_pos: list                      # per cloud: [n_ps, 3] root units or None
    ps_L: list                        # per cloud: [n_ps, n_freq] or None
    n_bg: list                        # per cloud: packages per frequency
    n_ps: list
    seed: int = 1
    extra: dict = field(default_factory=dict)


def config_c1(n_packages: int = 100_000) -> Workload:
    """32^3 uniform cube, centre-to-edge tau_ext = 1 (kappa_ext h = 1/16),
    albedo 0.5, isotropic scattering, unit isotropic background, one
    frequency, seed 1."""
    cl = regular(np.ones((32, 32, 32), np.float32), ell=1.0)
    nu = np.array([NU_1UM])
    dust = Dust(nu, np.array([1.0 / 32.0]), np.array([1.0 / 32.0]), np.array([0.0]))
    return Workload("c1_uniform32_1nu", [cl], dust, [np.array([1.0])], [None], [None],
                    [n_packages], [0], seed=1)


def config_c2(n: int = 128, n_freq: int = 64, n_packages: int = 1_000_000,
              side_pc: float = 1.0, tau_1um: float = 5.0, seed_field: int = 2) -> Workload:
    """n^3 lognormal cloud (sigma_lnrho 1.5, P(k) ~ k^-3.5), 64 log-spaced
    frequencies 3e11-3e15 Hz, kappa ~ nu^2 with a smooth albedo, HG g = 0.5,
    3-blackbody background, mean-density centre-to-face tau_ext(1 um) = 5."""
    rho = lognormal_density(n, seed_field, 1.5, -3.5).astype(np.float32)
    ell = side_pc * PC_CM / n
    cl = regular(rho, ell=ell)
    nu = frequency_grid(n_freq)
    kext_1um = tau_1um / ((n / 2) * ell * 1.0)
    dust = power_law_dust(nu, kext_1um)
    return Workload(f"c2_lognormal{n}_{n_freq}nu", [cl], dust, [diluted_blackbodies(nu)], [None],
                    [None], [n_packages], [0], seed=1)


def config_c3(root_n: int = 64, max_refine: int = 3, n_freq: int = 64, sigma: float = 1.5,
              threshold: float = 10.0, tau_peak_1um: float = 100.0, side_pc: float = 0.5,
              n_bg: int = 1_000_000, n_ps: int = 1_000_000, L_bol: float = 1e37,
              seed_field: int = 3, rule: str = "max") -> Workload:
    """Octree cloud: lognormal GRF (sigma_lnrho 1.5, P(k) ~ k^-3.5) at
    (root_n 2^max_refine)^3, a cell refined where the fine-grid density inside
    it exceeds 10x the global mean (about 4.9e6 cells for the 64^3 root with
    3 refinement levels); peak centre optical depth ~100 at 1 um (max over the
    six axis rays from the centre); 3 blackbody point sources (1e4 K) plus the
    3-blackbody background."""
    N = root_n << max_refine
    fine = lognormal_density(N, seed_field, sigma, -3.5)
    ell = side_pc * PC_CM / root_n
    cl = octree_from_fine(fine, root_n, max_refine, threshold, ell=ell, rule=rule)
    # normalise the opacity on the fine field: max over 6 axis rays of tau
    c = N // 2
    rays = [fine[c, c, c:].sum(), fine[c, c, :c].sum(), fine[c, c:, c].sum(),
            fine[c, :c, c].sum(), fine[c:, c, c].sum(), fine[:c, c, c].sum()]
    fine_cell = ell / (1 << max_refine)
    kext_1um = tau_peak_1um / (max(rays) * fine_cell)
    nu = frequency_grid(n_freq)
    dust = power_law_dust(nu, kext_1um)
    pos = np.array([[0.5, 0.5, 0.5], [0.3, 0.6, 0.4], [0.7, 0.35, 0.65]]) * root_n
    L = np.stack([stellar_luminosity(nu, 1e4, L_bol) for _ in range(3)])
    return Workload(f"c3_octree{root_n}r{max_refine}_{n_freq}nu", [cl], dust,
                    [diluted_blackbodies(nu)], [pos], [L], [n_bg], [n_ps], seed=1)


def config_c5(n_clouds: int = 64, n_freq: int = 32, seed: int = 5, sizes=None,
              base_packages: int = 100_000, L_bol: float = 1e36) -> Workload:
    """Uneven batch: clouds of side N in {32, 48, ..., 128} (seeded), tau(1um)
    ~ logU(0.5, 100), 1-3 point sources each, 32 frequencies, packages per
    cloud round(1e5 (N/32)^1.66)."""
    rng = np.random.default_rng(seed)
    nu = frequency_grid(n_freq)
    if sizes is None:
        sizes = rng.choice(np.arange(32, 129, 16), size=n_clouds)
    clouds, bg, pos, Ls, nbg, nps = [], [], [], [], [], []
    taus = np.exp(rng.uniform(np.log(0.5), np.log(100.0), size=len(sizes)))
    for ci, N in enumerate(sizes):
        N = int(N)
        rho = lognormal_density(N, 1000 + ci, float(rng.uniform(1.0, 2.0)), -3.5).astype(np.float32)
        ell = 1.0 * PC_CM / N
        clouds.append(regular(rho, ell=ell))
        bg.append(diluted_blackbodies(nu))
        k = int(rng.integers(1, 4))
        pos.append(rng.uniform(0.2, 0.8, size=(k, 3)) * N)
        Ls.append(np.stack([stellar_luminosity(nu, 1e4, L_bol) for _ in range(k)]))
        npk = int(round(base_packages * (N / 32) ** 1.66))
        nbg.append(npk)
        nps.append(npk)
    # one opacity table shared by the batch; per-cloud optical depth enters
    # through the density scale
    dust = power_law_dust(nu, 1.0)
    for ci, cl in enumerate(clouds):
        N = cl.nx
        scale = taus[ci] / ((N / 2) * cl.ell * 1.0)
        cl.rho = (cl.rho * scale).astype(np.float32)
    return Workload(f"c5_batch{len(sizes)}_{n_freq}nu", clouds, dust, bg, pos, Ls, nbg, nps,
                    seed=1, extra=dict(sizes=np.asarray(sizes), taus=taus))


def config_c4(seeds, side: int = 64, n_freq: int = 64, side_pc: float = 0.15, n_bg: int = 200_000,
              n_ps: int = 200_000, tau_range=(1000.0, 5000.0), L_range=(1e38, 5e38)) -> Workload:
    """Clouds of the learned-seed set, one per seed, in one workload that
    shares a single opacity table: hot-core clouds after the setup of the
    paper's convergence test (Sect. 3.3: a cloud shrunk and made denser, with
    an internal source heating the nearest cells to hundreds of K, so that
    dust re-emission matters over a large volume and the temperatures
    converge only after many iterations).  Per seed, all draws from
    numpy.random.default_rng(10_000 + seed): side^3 lognormal GRF (field seed
    = seed, sigma_lnrho ~ U(1, 2), P(k) ~ k^-3.5); mean-density centre-to-face
    tau_ext(1 um) ~ logU(tau_range), set through the density scale (the
    opacity is normalised so that unit density gives tau = 1); 1-2 blackbody
    point sources (1e4 K) with total luminosity ~ logU(L_range) erg/s,
    shared equally, at uniform positions in the inner 30 % of the box; the
    3-blackbody background; side_pc parsecs per side."""
    seeds = [int(s) for s in np.atleast_1d(seeds)]
    nu = frequency_grid(n_freq)
    ell = side_pc * PC_CM / side
    dust = power_law_dust(nu, 1.0 / ((side / 2) * ell))
    clouds, pos, Ls, extra = [], [], [], []
    for seed in seeds:
        rng = np.random.default_rng(10_000 + seed)
        sigma = float(rng.uniform(1.0, 2.0))
        tau = float(np.exp(rng.uniform(np.log(tau_range[0]), np.log(tau_range[1]))))
        k = int(rng.integers(1, 3))
        p = rng.uniform(0.35, 0.65, size=(k, 3)) * side
        L_tot = float(np.exp(rng.uniform(np.log(L_range[0]), np.log(L_range[1]))))
        rho = lognormal_density(side, seed, sigma, -3.5)
        clouds.append(regular((rho * tau).astype(np.float32), ell=ell))
        pos.append(p)
        Ls.append(np.stack([stellar_luminosity(nu, 1e4, L_tot / k) for _ in range(k)]))
        extra.append(dict(seed=seed, sigma=sigma, tau=tau, n_sources=k, L=L_tot))
    bg = diluted_blackbodies(nu)
    return Workload(f"c4_hotcore{side}_{len(seeds)}clouds", clouds, dust, [bg] * len(seeds), pos, Ls,
                    [n_bg] * len(seeds), [n_ps] * len(seeds), seed=1, extra=dict(clouds=extra))
