"""FP64 physics of the equilibrium-dust path (test infrastructure only).

Plain NumPy/SciPy definitions, one function per quantity, in the order the
method uses them (Juvela 2019, arXiv:1812.06632, Sect. 2.1.1: the frequency
integral of absorbed energy is gathered on the device; a separate kernel
solves the equilibrium temperature of each cell; with a reference/constant
field the constant sources are simulated once, Sect. 2.1.2).

Units: cgs.  Densities rho are in arbitrary "density units"; opacities kappa
are cross sections per density unit (rho * kappa is an inverse length in cm);
a cell of hierarchy level L (0-based) has side ell * 2^-L for root-cell side
ell (cm).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

# CODATA 2018 exact SI-defined constants, in cgs
H_PLANCK = 6.62607015e-27      # erg s
K_BOLTZ = 1.380649e-16         # erg / K
C_LIGHT = 2.99792458e10        # cm / s
W_UNIT = 2.0 ** 31             # fixed-point units of one package's initial weight

T_MIN = 2.7                    # K: temperature of cells that absorb nothing
T_MAX = 3000.0                 # K: upper end of the solver's range


def planck_nu(nu, T):
    """B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1)  [erg/s/cm^2/Hz/sr]."""
    nu = np.asarray(nu, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    x = H_PLANCK * nu / (K_BOLTZ * T)
    with np.errstate(over="ignore"):
        return (2.0 * H_PLANCK * nu ** 3 / C_LIGHT ** 2) / np.expm1(x)


def dplanck_dT(nu, T):
    """dB_nu/dT."""
    nu = np.asarray(nu, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    x = H_PLANCK * nu / (K_BOLTZ * T)
    with np.errstate(over="ignore", invalid="ignore"):
        em1 = np.expm1(x)
        val = (2.0 * H_PLANCK * nu ** 3 / C_LIGHT ** 2) * (x / T) * (em1 + 1.0) / (em1 * em1)
    return np.nan_to_num(val, nan=0.0, posinf=0.0)


def trapezoid_weights(nu):
    """Trapezoid-rule weights w_nu on the frequency nodes (sum_nu w f(nu) ~ int f dnu)."""
    nu = np.asarray(nu, dtype=np.float64)
    w = np.zeros_like(nu)
    if nu.size == 1:
        w[0] = 1.0
        return w
    d = np.diff(nu)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return w


def emission_integral(T, nu, kabs):
    """E(T) = 4 pi sum_nu w_nu kabs(nu) B_nu(T): power emitted per unit of rho*V."""
    w = trapezoid_weights(nu)
    return 4.0 * np.pi * float(np.sum(w * np.asarray(kabs, np.float64) * planck_nu(nu, T)))


def temperature(A, nu, kabs, t_min=T_MIN, t_max=T_MAX, rtol=1e-13):
    """Equilibrium temperature: root of E(T) = A (Brent's method).  A at or
    below E(t_min) (in particular no absorption) gives t_min; above E(t_max)
    gives t_max."""
    A = float(A)
    e_lo = emission_integral(t_min, nu, kabs)
    e_hi = emission_integral(t_max, nu, kabs)
    if not A > e_lo:
        return t_min
    if A >= e_hi:
        return t_max
    return brentq(lambda T: emission_integral(T, nu, kabs) - A, t_min, t_max,
                  xtol=1e-14, rtol=rtol, maxiter=500)


def temperatures(A, nu, kabs, **kw):
    return np.array([temperature(a, nu, kabs, **kw) for a in np.asarray(A).ravel()])


def cell_volumes(grid, ell):
    """Volume (cm^3) of every cell of an oracle.Grid with root-cell side ell."""
    lv = grid.level_of()
    return (ell * np.ldexp(1.0, -lv)) ** 3


def absorbed_power(tally, e_unit, nu, rho, volume, A_in=None):
    """Absorbed power per unit rho*V (Sect. 2.1.1's frequency integral):
    A_c = A_in + sum_nu w_nu e_unit(nu) tally[nu, c] / (rho_c V_c).
    ``tally`` is int64 [n_freq, n_cells]; ``e_unit[nu]`` the energy (erg/s/Hz)
    of one fixed-point unit.  Cells with rho = 0 (and parents) get A_in."""
    tally = np.asarray(tally)
    w = trapezoid_weights(nu)
    acc = np.zeros(tally.shape[1], np.float64)
    for k in range(tally.shape[0]):
        acc += (w[k] * float(e_unit[k])) * tally[k].astype(np.float64)
    rv = np.asarray(rho, np.float64) * np.asarray(volume, np.float64)
    out = np.zeros_like(acc) if A_in is None else np.array(A_in, np.float64, copy=True)
    ok = rv > 0
    out[ok] += acc[ok] / rv[ok]
    return out


def background_package_energy(I_nu, nx, ny, nz, ell, n_packages):
    """Energy per unit of weight of a background package.  An isotropic
    intensity I_nu outside the box sends pi I_nu per unit area through every
    face, so the packages share pi I_nu S (S the box surface); one package
    starts with 2^31 units."""
    S = 2.0 * (nx * ny + ny * nz + nz * nx) * ell * ell
    return np.pi * np.asarray(I_nu, np.float64) * S / n_packages / W_UNIT


def point_package_energy(L_nu_total, n_packages):
    """Energy per unit of weight of a point-source package: the sources'
    total luminosity L_nu (erg/s/Hz) shared by n_packages."""
    return np.asarray(L_nu_total, np.float64) / n_packages / W_UNIT


def point_source_cdf(L_nu):
    """Cumulative luminosity fractions per frequency, [n_freq, n_ps], FP32,
    used to pick the source of a package (last entry forced to 1)."""
    L = np.asarray(L_nu, np.float64)          # [n_ps, n_freq]
    tot = L.sum(axis=0)
    cdf = np.cumsum(L, axis=0) / np.where(tot > 0, tot, 1.0)
    cdf[-1, :] = 1.0
    return cdf.T.astype(np.float32)


def dust_luminosity(T, rho, volume, kabs_nu, nu):
    """L_c(nu) = 4 pi rho_c V_c kabs(nu) B_nu(T_c) of the given cells (erg/s/Hz)."""
    return 4.0 * np.pi * np.asarray(rho, np.float64) * np.asarray(volume, np.float64) \
        * float(kabs_nu) * planck_nu(nu, np.asarray(T, np.float64))


def dust_weights(L, n_per_cell):
    """Fixed-point initial weights of dust packages at one frequency: every
    cell sends n_per_cell packages; W_c = rint(2^31 L_c / max L), and one unit
    then carries e_unit = (max L / n_per_cell) / 2^31.  Returns (W uint64, e_unit)."""
    L = np.asarray(L, np.float64)
    Lmax = float(L.max()) if L.size else 0.0
    if not Lmax > 0:
        return np.zeros(L.shape, np.uint64), 0.0
    W = np.rint((L / Lmax) * W_UNIT).astype(np.uint64)
    return W, Lmax / n_per_cell / W_UNIT


def temperature_ali(A, A_self, T_old, nu, kabs, beta_max=0.99, **kw):
    """Accelerated update with the diagonal (one-cell) operator: the part of
    A that the cell absorbed from its own emission, A_self, is assumed to
    scale with its emission, A_self(T) = beta E(T) with beta = A_self /
    E(T_old) (at most beta_max); T solves E(T) (1 - beta) = A - A_self."""
    E_old = emission_integral(T_old, nu, kabs)
    beta = min(beta_max, A_self / E_old) if E_old > 0 else 0.0
    beta = max(beta, 0.0)
    return temperature((A - A_self) / (1.0 - beta), nu, kabs, **kw)


def weighted_dust_sampling(u, e_unit_uniform, n_total, cap):
    """Emission-weighted dust sampling (paper Sect. 3.2: packages per cell in
    proportion to the cell's luminosity, at most `cap` from any cell), built
    from the uniform weights u_c = rint(2^31 L_c / max L) of one frequency:
      S = sum u_c (integer),
      n_c = 0 if u_c = 0 else min(cap, ceil(N u_c / S)),
      E_ref = max(S / N, 2^31 / cap)  (in units of max L / 2^31),
      W_c = rint((u_c / n_c) / E_ref * 2^31)  (<= 2^31),
      one fixed-point unit carries e_unit_uniform * E_ref / 2^31.
    Returns (n uint64, exclusive prefix uint64 [n_leaf + 1], W uint64, e_unit)."""
    u = np.asarray(u, np.uint64)
    S = int(u.sum(dtype=np.uint64))
    n = np.zeros(u.shape, np.uint64)
    W = np.zeros(u.shape, np.uint64)
    if S == 0:
        return n, np.zeros(u.size + 1, np.uint64), W, 0.0
    uf = u.astype(np.float64)
    nz = u > 0
    n[nz] = np.minimum(float(cap), np.ceil(float(n_total) * uf[nz] / float(S))).astype(np.uint64)
    E_ref = max(float(S) / float(n_total), W_UNIT / float(cap))
    W[nz] = np.rint((uf[nz] / n[nz].astype(np.float64)) / E_ref * W_UNIT).astype(np.uint64)
    prefix = np.zeros(u.size + 1, np.uint64)
    prefix[1:] = np.cumsum(n, dtype=np.uint64)
    return n, prefix, W, float(e_unit_uniform) * E_ref / W_UNIT


def weighted_dust_reweight(u, e_unit_uniform, prefix):
    """Weights for an existing (frozen) allocation n_c = prefix[c+1] - prefix[c]
    at new temperatures: E_ref = max over cells with n_c > 0 of u_c / n_c,
    W_c = rint((u_c / n_c) / E_ref 2^31), e_unit = e_unit_uniform E_ref / 2^31.
    Frozen counts keep every package's id -> cell map, so iterations with
    frozen random numbers follow the same paths."""
    u = np.asarray(u, np.uint64)
    pre = np.asarray(prefix, np.uint64)
    n = (pre[1:] - pre[:-1]).astype(np.float64)
    W = np.zeros(u.shape, np.uint64)
    ok = n > 0
    if not ok.any():
        return W, 0.0
    q = u[ok].astype(np.float64) / n[ok]
    E_ref = float(q.max())
    if not E_ref > 0:
        return W, 0.0
    W[ok] = np.rint(q / E_ref * W_UNIT).astype(np.uint64)
    return W, float(e_unit_uniform) * E_ref / W_UNIT


# ---------------------------------------------------------------------------
# Reference field (Sect. 2.1.2; Sects. 3.4, 3.6 and 4.1).  The stored
# reference is the absorbed power A_ref of each cell, the package-weighted
# mean of the dust-absorption estimates of the iterations done (fresh random
# numbers each iteration), so its noise falls with the number of iterations
# and early iterations with few packages count less; T comes from
# A_const + A_ref ("mean" reading).  The "difference" variant traces only the
# change of the emission against a reference emission L_ref (also a running
# mean) and takes T from A_const + A_ref + the traced change.
# ---------------------------------------------------------------------------
def package_schedule(n_first, n_last, n_iter):
    """Dust packages per frequency of iterations 1..n_iter, log n growing
    linearly (Sect. 3.6): n_k = rint(n_first (n_last / n_first)^((k-1)/(n_iter-1)))."""
    k = np.arange(n_iter, dtype=np.float64)
    if n_iter == 1:
        return np.array([int(n_last)], np.uint64)
    ratio = float(n_last) / float(n_first)
    return np.rint(float(n_first) * ratio ** (k / float(n_iter - 1))).astype(np.uint64)


def reference_weights(n):
    """w_k = n_k / sum_{j <= k} n_j: the step of the running package-weighted mean."""
    n = np.asarray(n, np.float64)
    return n / np.cumsum(n)


def reference_delta(L, L_ref, w):
    """Emission change of one frequency, d = L - L_ref (per leaf), as weights
    of the emission-weighted sampler: m = max |d|, u = rint(|d| / m 2^31),
    neg = d < 0, one unit of u carrying e_uni = m / 2^31 (one package per
    cell).  The reference moves to L_ref + w d.  Returns (u, neg, e_uni, L_ref')."""
    L = np.asarray(L, np.float64)
    L_ref = np.asarray(L_ref, np.float64)
    d = L - L_ref
    a = np.abs(d)
    m = float(a.max()) if a.size else 0.0
    u = np.zeros(L.shape, np.uint64)
    if m > 0:
        u = np.rint((a / m) * W_UNIT).astype(np.uint64)
    return u, d < 0, m / W_UNIT, L_ref + w * d


def split_allocation(W, neg):
    """Weights of the packages from cells whose emission rose (first) and fell
    (second); the allocation (prefix) is shared."""
    W = np.asarray(W, np.uint64)
    z = np.zeros_like(W)
    return np.where(neg, z, W), np.where(neg, W, z)


def reference_update(A_ref, A_d, w):
    """A_ref + w (A_d - A_ref): the running mean moved towards the estimate
    A_d of this iteration (the full dust absorption in the "mean" reading,
    A_ref + the traced change in the "difference" variant)."""
    A_ref = np.asarray(A_ref, np.float64)
    return A_ref + w * (np.asarray(A_d, np.float64) - A_ref)
