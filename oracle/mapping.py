"""FP64 oracle of the surface-brightness maps (test infrastructure only).

For every pixel the ray x(t) = o + t d is cut at every plane where any cell
of the hierarchy can begin or end (x = m h_min for the finest cell side
h_min = 2^-(levels-1), same for y and z); between consecutive cuts the ray
lies in one leaf, found by descending from the root at the segment's
midpoint.  Along each segment of extinction depth dtau the intensity gains
(kabs/kext) B_nu(T) (1 - e^-dtau) e^-tau_front (paper Sect. 2.1.1: maps from
the solved temperatures), and the background arrives attenuated by the total
depth.
"""
from __future__ import annotations

import numpy as np

from . import physics as P


def _leaf_at(grid, point):
    """Leaf containing a root-unit point (descending from its root cell)."""
    i = [min(max(int(np.floor(point[a])), 0), n - 1) for a, n in enumerate((grid.nx, grid.ny, grid.nz))]
    c = i[0] + grid.nx * (i[1] + grid.ny * i[2])
    lo = np.array(i, np.float64)
    h = 1.0
    while grid.child[c] >= 0:
        h /= 2.0
        b = [(point[a] >= lo[a] + h) for a in range(3)]
        lo = lo + h * np.array(b, np.float64)
        c = grid.child[c] + (b[0] | (b[1] << 1) | (b[2] << 2))
    return c


def frame(direction, up):
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    e1 = np.cross(np.asarray(up, np.float64), d)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    return d, e1, e2


def ray_map(grid, T, kabs_root, ksca_root, nu, direction, up, npx, npy, pix, center, I_bg=0.0):
    """Map [npy, npx]; kabs_root, ksca_root = cross sections x root-cell side."""
    d, e1, e2 = frame(direction, up)
    n = np.array([grid.nx, grid.ny, grid.nz], np.float64)
    hmin = 2.0 ** -(grid.n_levels - 1)
    kext = kabs_root + ksca_root
    ratio = kabs_root / kext if kext > 0 else 0.0
    out = np.zeros((npy, npx))
    for py in range(npy):
        for px in range(npx):
            o = np.asarray(center, np.float64) + ((px + 0.5) - npx / 2) * pix * e1 + ((py + 0.5) - npy / 2) * pix * e2
            t0, t1 = -np.inf, np.inf
            for a in range(3):
                if d[a] == 0.0:
                    if o[a] < 0 or o[a] > n[a]:
                        t0, t1 = 1.0, 0.0
                    continue
                ta, tb = sorted(((0.0 - o[a]) / d[a], (n[a] - o[a]) / d[a]))
                t0, t1 = max(t0, ta), min(t1, tb)
            I, tau = 0.0, 0.0
            if t0 < t1:
                cuts = [t0, t1]
                for a in range(3):
                    if d[a] == 0.0:
                        continue
                    xa, xb = sorted((o[a] + t0 * d[a], o[a] + t1 * d[a]))
                    m = np.arange(np.ceil(xa / hmin), np.floor(xb / hmin) + 1) * hmin
                    cuts.extend(((m - o[a]) / d[a]).tolist())
                cuts = np.unique(np.clip(cuts, t0, t1))
                for ta, tb in zip(cuts[:-1], cuts[1:]):
                    if tb - ta <= 0:
                        continue
                    c = _leaf_at(grid, o + 0.5 * (ta + tb) * d)
                    dtau = float(grid.rho[c]) * kext * (tb - ta)
                    if dtau > 0:
                        B = float(P.planck_nu(nu, float(T[c])))
                        I += ratio * B * (-np.expm1(-dtau)) * np.exp(-tau)
                        tau += dtau
            out[py, px] = I + I_bg * np.exp(-tau)
    return out
