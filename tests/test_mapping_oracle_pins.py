"""Pins of the FP64 map oracle: closed forms for a uniform cube (axis and
oblique views), and invariance under refinement of a uniform cloud."""
import numpy as np

import oracle
from oracle import mapping as M
from oracle import physics as P
from paper_1812_06632_gb300 import inputs as I


def _grid(cl):
    return oracle.Grid(cl.nx, cl.ny, cl.nz, cl.level_start, cl.rho, cl.child, cl.parent)


def _chord(o, d, n):
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        if d[a] == 0:
            if not (0 <= o[a] <= n[a]):
                return 0.0
            continue
        ta, tb = sorted(((0 - o[a]) / d[a], (n[a] - o[a]) / d[a]))
        t0, t1 = max(t0, ta), min(t1, tb)
    return max(0.0, t1 - t0)


def test_uniform_cube_closed_form_axis_and_oblique():
    n, rho, ka, ks, T, nu = 6, 2.0, 0.07, 0.05, 40.0, 3e12
    cl = I.regular(np.full((n, n, n), rho, np.float32))
    Tc = np.full(cl.n_cells, T)
    B = float(P.planck_nu(nu, T))
    for direction in ([0, 0, 1], [0.3, -0.5, 0.8]):
        img = M.ray_map(_grid(cl), Tc, ka, ks, nu, direction, [0, 1, 0], 9, 7, 0.9, [3.0, 3.0, 3.0], I_bg=0.5)
        d, e1, e2 = M.frame(direction, [0, 1, 0])
        for py in range(7):
            for px in range(9):
                o = np.array([3.0, 3, 3]) + ((px + 0.5) - 4.5) * 0.9 * e1 + ((py + 0.5) - 3.5) * 0.9 * e2
                L = _chord(o - 100 * d, d, [n, n, n])
                tau = rho * (ka + ks) * L
                exp_I = ka / (ka + ks) * B * (-np.expm1(-tau)) + 0.5 * np.exp(-tau)
                assert abs(img[py, px] - exp_I) <= 1e-12 * max(1.0, exp_I)


def test_refined_uniform_cloud_gives_the_same_map():
    n = 4
    base = I.regular(np.full((n, n, n), 1.5, np.float32))
    ref = I.refine_cells(base, [0, 5, 21, 42, 63])
    ref = I.refine_cells(ref, [ref.level_start[1] + 3, ref.level_start[1] + 17])
    T0 = np.full(base.n_cells, 25.0)
    T1 = np.full(ref.n_cells, 25.0)
    args = (0.2, 0.1, 1e13, [0.2, 0.7, -0.4], [0, 0, 1], 8, 8, 0.6, [2.0, 2.0, 2.0])
    a = M.ray_map(_grid(base), T0, *args)
    b = M.ray_map(_grid(ref), T1, *args)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_temperature_structure_shows_in_the_map():
    """A single hot cell in a thin cloud adds exactly its own emission."""
    n = 5
    cl = I.regular(np.full((n, n, n), 1e-3, np.float32))
    T = np.full(cl.n_cells, 10.0)
    hot = 2 + n * (2 + n * 2)
    T[hot] = 100.0
    nu, ka = 3e12, 0.5
    img = M.ray_map(_grid(cl), T, ka, 0.0, nu, [0, 0, 1], [0, 1, 0], 5, 5, 1.0, [2.5, 2.5, 2.5])
    col = img[2, 2]
    other = img[0, 0]
    dtau = float(np.float32(1e-3)) * ka            # the grid stores FP32 densities
    gain = (float(P.planck_nu(nu, 100.0)) - float(P.planck_nu(nu, 10.0))) * (-np.expm1(-dtau)) * np.exp(-2 * dtau)
    assert abs((col - other) / gain - 1) < 1e-9
