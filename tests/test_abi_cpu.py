"""C-ABI checks that need no GPU: every symbol declared in include/soc.h is
exported by libsoc.so, and the host-side grid validation accepts the paper's
layout and rejects malformed grids."""
import os
import re

import numpy as np
import pytest

from paper_1812_06632_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "soc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(soc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(libsoc):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(libsoc.lib, n), n
    assert set(libsoc.EXPORTS) == set(names)


def _v(libsoc, cl, **over):
    args = dict(nx=cl.nx, ny=cl.ny, nz=cl.nz, cells_per_level=cl.cells_per_level(), rho=cl.rho,
                first_child=cl.child, parent=cl.parent if cl.parent.size else None, ell=cl.ell)
    args.update(over)
    return libsoc.validate_grid(**args)


def test_valid_grids(libsoc):
    reg = I.regular(np.ones((3, 4, 5), np.float32))
    assert _v(libsoc, reg)[0] == 0
    oc = I.config_c3(root_n=8, max_refine=2, threshold=3.0).clouds[0]
    assert oc.n_levels == 3
    assert _v(libsoc, oc)[0] == 0
    # the paper's encoding: links as negative densities, no child array
    assert _v(libsoc, oc, rho=oc.paper_encoding(), first_child=None)[0] == 0
    # parent array may be omitted
    assert _v(libsoc, oc, parent=None)[0] == 0


@pytest.mark.parametrize("case", ["link_range", "link_level", "two_parents", "orphan", "nan", "neg",
                                  "parent_mismatch", "cpl", "bad_paper_link", "ell"])
def test_malformed_grids_rejected(libsoc, case):
    oc = I.config_c3(root_n=8, max_refine=2, threshold=3.0).clouds[0]
    child, rho, parent = oc.child.copy(), oc.rho.copy(), oc.parent.copy()
    over = {}
    refined = np.nonzero(child >= 0)[0]
    leaves = np.nonzero(child < 0)[0]
    if case == "link_range":
        child[refined[0]] = oc.n_cells + 8
    elif case == "link_level":                      # points into its own level
        child[refined[0]] = 0
    elif case == "two_parents":
        child[refined[1]] = child[refined[0]]
    elif case == "orphan":
        child[refined[-1]] = -1
    elif case == "nan":
        rho[leaves[3]] = np.nan
    elif case == "neg":
        rho[leaves[5]] = -1.0
    elif case == "parent_mismatch":
        parent[0] = parent[1]
    elif case == "cpl":
        over["cells_per_level"] = oc.cells_per_level() + np.array([0, 1, 0])
    elif case == "bad_paper_link":
        rho = oc.paper_encoding()
        rho[refined[0]] = -float(child[refined[0]]) - 0.5
        child = None
    elif case == "ell":
        over["ell"] = 0.0
    st, msg = _v(libsoc, oc, rho=rho, first_child=child, parent=parent, **over)
    assert st in (-1, -2), (case, st, msg)
    assert msg and msg != "ok"


def test_large_grid_checks_report_the_first_bad_cell(libsoc):
    """Grids of 2^18 cells and more are checked by several host threads: the
    error reported is still the one at the lowest cell index, and a planted
    error is found in whichever chunk it falls."""
    n = 64
    rho = np.random.default_rng(0).uniform(0.5, 2.0, n ** 3).astype(np.float32)
    reg = I.regular(rho.reshape(n, n, n))
    assert _v(libsoc, reg)[0] == 0
    for bad in (0, 70_000, n ** 3 - 1):
        r = reg.rho.copy()
        r[bad] = np.nan
        st, msg = _v(libsoc, reg, rho=r)
        assert st == -2 and f"leaf {bad} " in msg, msg
    r = reg.rho.copy()
    r[250_000] = -1.0
    r[90_000] = np.inf
    st, msg = _v(libsoc, reg, rho=r)
    assert st == -2 and "leaf 90000 " in msg, msg


def test_large_octree_checks(libsoc):
    """An octree of more than 2^18 cells (threaded checks): valid as built;
    two parents for one octet, an orphan octet and a bad leaf are found."""
    oc = I.config_c3(root_n=32, max_refine=2, threshold=2.0).clouds[0]
    assert oc.n_cells >= 1 << 18 and oc.n_levels == 3
    assert _v(libsoc, oc)[0] == 0
    assert _v(libsoc, oc, rho=oc.paper_encoding(), first_child=None, parent=None)[0] == 0
    refined = np.nonzero(oc.child >= 0)[0]
    leaves = np.nonzero(oc.child < 0)[0]
    root_refined = refined[refined < oc.nx * oc.ny * oc.nz]     # two far-apart cells of one level
    child = oc.child.copy()
    child[root_refined[-1]] = child[root_refined[0]]
    st, msg = _v(libsoc, oc, first_child=child, parent=None)
    assert st == -2 and "two parents" in msg, msg
    child = oc.child.copy()
    child[refined[len(refined) // 2]] = -1
    st, msg = _v(libsoc, oc, first_child=child, parent=None)
    assert st == -2, msg
    rho = oc.rho.copy()
    rho[leaves[-1]] = -3.0
    st, msg = _v(libsoc, oc, rho=rho)
    assert st == -2 and f"leaf {leaves[-1]} " in msg, msg


def test_weight_unit_agrees_across_header_binding_and_oracle(libsoc):
    """The fixed-point unit of one package is the same constant in the C-ABI
    header, the binding, the test helpers and the oracle (C and FP64 parts)."""
    import oracle
    from oracle import physics as P
    from parity_helpers import W_UNIT as helper_unit
    src = open(os.path.join(ROOT, "include", "soc.h")).read()
    m = re.search(r"#define\s+SOC_W_UNIT\s+(\d+)ull", src)
    header_unit = int(m.group(1))
    assert header_unit == libsoc.W_UNIT == helper_unit == oracle.W_UNIT == int(P.W_UNIT) == 1 << 31


def test_binding_fails_loudly_without_the_library(tmp_path):
    """With its library missing the binding raises at import: there is no
    CPU fallback to fall through to."""
    import subprocess
    import sys
    env = dict(os.environ, SOC_LIB=str(tmp_path / "absent" / "libsoc.so"))
    r = subprocess.run([sys.executable, "-c", "import paper_1812_06632_gb300.soc"], cwd=ROOT, env=env,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "missing" in r.stderr


def test_product_path_never_touches_the_oracle():
    """No file of the package or of include/ imports, links or loads the
    oracle (only tests/, smoke() and bench.py's CPU legs may)."""
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|liboracle|soc_oracle", re.M)
    hits = []
    for d in ("paper_1812_06632_gb300", "include"):
        for dp, _, fs in os.walk(os.path.join(ROOT, d)):
            if "_build" in dp or "__pycache__" in dp:
                continue
            for f in fs:
                if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                    if pat.search(open(os.path.join(dp, f), errors="replace").read()):
                        hits.append(os.path.join(dp, f))
    assert not hits, hits


def test_binding_refuses_host_and_strided_tensors(libsoc):
    """Device-pointer arguments must be dense CUDA tensors: anything else is
    refused on the host, before a kernel could address the wrong memory."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        libsoc._t_ptr(torch.zeros(4))
    assert libsoc._t_ptr(None) is None


def test_learned_seed_entry_points_reject_bad_arguments_on_the_host(libsoc):
    """The network helpers check their arguments before any CUDA call, as
    include/soc.h states (SOC_ERR_ARG = -1): null pointers, sizes, a NaN
    factor, and four features without the iterate before the previous one.
    The device pointers given are never dereferenced on these paths."""
    import ctypes as C
    ERR_ARG = -1
    fake = C.c_void_p(0x1000)                      # a non-null device address, never touched here
    f = libsoc.lib.soc_nn_scale_add
    assert f(None, fake, 10, C.c_float(1.0), None) == ERR_ARG
    assert f(fake, None, 10, C.c_float(1.0), None) == ERR_ARG
    assert f(fake, fake, 0, C.c_float(1.0), None) == ERR_ARG
    assert f(fake, fake, 10, C.c_float(float("nan")), None) == ERR_ARG
    norm = np.ascontiguousarray([0.0, 1.0] * 4, np.float64)
    nptr = norm.ctypes.data_as(C.c_void_p)
    g = libsoc.lib.soc_nn_seed_features
    # (T, T_prev, T_prev2, rho, n, norm, n_features, x, stream)
    assert g(fake, fake, None, fake, 10, nptr, 4, fake, None) == ERR_ARG      # four features need T_prev2
    assert g(fake, None, None, fake, 10, nptr, 3, fake, None) == ERR_ARG      # three need T_prev
    assert g(fake, fake, fake, fake, 10, nptr, 5, fake, None) == ERR_ARG      # 2 to 4 features
    assert g(fake, fake, fake, None, 10, nptr, 2, fake, None) == ERR_ARG      # rho
    bad = np.ascontiguousarray([0.0, 1.0, 0.0, 1.0, 0.0, 0.0], np.float64)   # a zero width
    assert g(fake, fake, None, fake, 10, bad.ctypes.data_as(C.c_void_p), 3, fake, None) == ERR_ARG
