"""CPU oracle for the SOC photon-package tracer and the equilibrium-temperature
update (Juvela 2019, arXiv:1812.06632, Sect. 2.1.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  The
product path (``paper_1812_06632_gb300``) never imports, links or executes
anything here, and this package imports nothing from the product path.

Three parts:

* ``soc_oracle.c`` (built with gcc into ``liboracle.so`` by :func:`build`):
  the tracer in the FP32 contract, one package at a time.  Its integer
  counters are what the CUDA tracer must reproduce bit for bit.
* ``soc_oracle64.c`` (``liboracle64.so``, :func:`trace64`): the same Monte
  Carlo, on the same random numbers, in FP64 with libm exp/log and real
  weights; it states how far the FP32 contract's counters are from an FP64
  run.
* :mod:`oracle.physics`: FP64 NumPy/SciPy definitions of the Planck law, the
  frequency quadrature, the normalisation of the counters to absorbed power
  and the equilibrium temperature (root-finding).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "soc_oracle.c")
_SRC64 = os.path.join(_HERE, "soc_oracle64.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_LIB64_PATH = os.path.join(_HERE, "_build", "liboracle64.so")
_lock = threading.Lock()
_lib = None
_lib64 = None

SRC_BACKGROUND, SRC_POINT, SRC_DUST = 0, 1, 2
W_UNIT = 1 << 31          # fixed-point units of one package's initial weight


def _gcc(out: str, srcs, force: bool) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fno-unsafe-math-optimizations", "-fPIC", "-shared", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile soc_oracle.c (FP32 contract flags: one rounding per written
    operation) and the FP64 oracle with gcc.  Returns the FP32 oracle's path."""
    _gcc(_LIB64_PATH, [_SRC64, _SRC], force)     # the FP64 tracer draws through the same Philox
    return _gcc(_LIB_PATH, [_SRC], force)


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("n_levels", C.c_int32), ("n_cells", C.c_int64),
                ("level_start", C.c_void_p), ("rho", C.c_void_p),
                ("child", C.c_void_p), ("parent", C.c_void_p)]


class _Item(C.Structure):
    _fields_ = [("source", C.c_int32), ("freq", C.c_int32), ("iteration", C.c_int32),
                ("cloud", C.c_int32), ("seed", C.c_uint64),
                ("kabs", C.c_float), ("ksca", C.c_float), ("g", C.c_float),
                ("w0", C.c_uint64), ("max_steps", C.c_uint32),
                ("n_ps", C.c_int32), ("ps_pos", C.c_void_p), ("ps_cdf", C.c_void_p),
                ("n_per_cell", C.c_uint32), ("n_leaf", C.c_int64),
                ("leaf", C.c_void_p), ("dust_w", C.c_void_p), ("dust_prefix", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("escaped", C.c_int64), ("capped", C.c_int64),
                ("steps", C.c_int64), ("emitted", C.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # SOC_ORACLE_LIB: a deliberately broken copy, for the mutation tests
            _lib = C.CDLL(os.environ.get("SOC_ORACLE_LIB") or build())
            P = C.c_void_p
            _lib.oracle_philox4x32_10.argtypes = [P, P, P]
            _lib.oracle_u01.argtypes = [C.c_uint32]
            _lib.oracle_u01.restype = C.c_float
            for n in ("oracle_one_minus_exp_v", "oracle_log_v"):
                getattr(_lib, n).argtypes = [P, P, C.c_int64]
            _lib.oracle_trace.argtypes = [C.POINTER(_Grid), C.POINTER(_Item), C.c_uint32,
                                          C.c_uint32, P, C.POINTER(_Stats), P, P]
            _lib.oracle_hg_samples.argtypes = [C.c_float, P, C.c_uint64, C.c_int64, P, P]
            _lib.oracle_trace_pencil.argtypes = [C.POINTER(_Grid), C.POINTER(_Item), P, P,
                                                 C.c_uint32, P, C.POINTER(_Stats)]
            _lib.oracle_trace_pencil.restype = C.c_uint32
        return _lib


class _Stats64(C.Structure):
    _fields_ = [("escaped", C.c_double), ("capped", C.c_int64),
                ("steps", C.c_int64), ("emitted", C.c_double)]


def lib64():
    global _lib64
    with _lock:
        if _lib64 is None:
            # SOC_ORACLE64_LIB: a deliberately broken copy, for the mutation tests
            path = os.environ.get("SOC_ORACLE64_LIB")
            if not path:
                build()
                path = _LIB64_PATH
            _lib64 = C.CDLL(path)
            _lib64.oracle64_trace.argtypes = [C.POINTER(_Grid), C.POINTER(_Item), C.c_uint32, C.c_uint32,
                                              C.c_void_p, C.POINTER(_Stats64), C.c_void_p]
        return _lib64


def _ptr(a):
    return None if a is None else a.ctypes.data


# --------------------------------------------------------------------------
# elementary pieces
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al. 2011) for counter[4], key[2]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(x: int) -> float:
    return float(lib().oracle_u01(int(x) & 0xFFFFFFFF))


def _vec(fn, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    fn(_ptr(x), _ptr(y), x.size)
    return y


def one_minus_exp(tau):
    """Contract 1 - exp(-tau), tau >= 0 (FP32)."""
    return _vec(lib().oracle_one_minus_exp_v, tau)


def log(u):
    """Contract ln(u) (FP32)."""
    return _vec(lib().oracle_log_v, u)


def hg_samples(g: float, d0, seed: int, n: int):
    d0 = np.ascontiguousarray(d0, dtype=np.float32)
    cosv = np.empty(n, np.float32)
    dout = np.empty((n, 3), np.float32)
    lib().oracle_hg_samples(C.c_float(g), _ptr(d0), C.c_uint64(seed), n, _ptr(cosv), _ptr(dout))
    return cosv, dout


# --------------------------------------------------------------------------
# tracer
# --------------------------------------------------------------------------
class Grid:
    """Level-ordered octree in the paper's layout (Sect. 2.1.1): root cells
    first, then every octet of level 2, then level 3, ...  ``child[c]`` is the
    index of the first cell of c's octet (-1 for a leaf); ``parent[k]`` is the
    parent of octet k (cells n_root + 8k .. n_root + 8k + 7)."""

    def __init__(self, nx, ny, nz, level_start, rho, child, parent):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.level_start = np.ascontiguousarray(level_start, dtype=np.int64)
        self.rho = np.ascontiguousarray(rho, dtype=np.float32)
        self.child = np.ascontiguousarray(child, dtype=np.int32)
        self.parent = np.ascontiguousarray(parent, dtype=np.int32)
        self.n_cells = int(self.rho.size)
        self.n_levels = int(self.level_start.size - 1)

    @property
    def n_root(self):
        return self.nx * self.ny * self.nz

    def leaves(self):
        return np.nonzero(self.child < 0)[0].astype(np.int32)

    def level_of(self):
        lv = np.zeros(self.n_cells, np.int32)
        for L in range(self.n_levels):
            lv[self.level_start[L]:self.level_start[L + 1]] = L
        return lv

    def _c(self):
        g = _Grid(self.nx, self.ny, self.nz, self.n_levels, self.n_cells,
                  _ptr(self.level_start), _ptr(self.rho), _ptr(self.child), _ptr(self.parent))
        return g


def trace(grid: Grid, *, source: int, kabs: float, ksca: float, g: float = 0.0,
          seed: int = 1, freq: int = 0, iteration: int = 0, cloud: int = 0,
          pid_lo: int = 0, n_packages: int, w0: int = W_UNIT, max_steps: int = 10_000_000,
          ps_pos=None, ps_cdf=None, n_per_cell: int = 1, leaf=None, dust_w=None,
          tally=None, want_steps: bool = False, self_tally=None, dust_prefix=None):
    """Trace packages pid_lo .. pid_lo + n_packages - 1 of one (source, freq)
    item.  ``kabs``/``ksca`` are per unit density and per root-cell length.
    ``self_tally`` (int64[n_cells], accumulated) receives the deposits dust
    packages make in their emission cell before they first leave it.
    Returns (tally int64[n_cells], stats dict, per-package steps or None)."""
    if tally is None:
        tally = np.zeros(grid.n_cells, np.int64)
    ps_pos_a = None if ps_pos is None else np.ascontiguousarray(ps_pos, np.float32).ravel()
    ps_cdf_a = None if ps_cdf is None else np.ascontiguousarray(ps_cdf, np.float32)
    leaf_a = None if leaf is None else np.ascontiguousarray(leaf, np.int32)
    dust_a = None if dust_w is None else np.ascontiguousarray(dust_w, np.uint64)
    pref_a = None if dust_prefix is None else np.ascontiguousarray(dust_prefix, np.uint64)
    it = _Item(source, freq, iteration, cloud, seed & (2**64 - 1),
               np.float32(kabs), np.float32(ksca), np.float32(g), w0, max_steps,
               0 if ps_cdf_a is None else ps_cdf_a.size, _ptr(ps_pos_a), _ptr(ps_cdf_a),
               n_per_cell, 0 if leaf_a is None else leaf_a.size, _ptr(leaf_a), _ptr(dust_a), _ptr(pref_a))
    st = _Stats()
    steps = np.zeros(n_packages, np.uint32) if want_steps else None
    gc = grid._c()
    lib().oracle_trace(C.byref(gc), C.byref(it), pid_lo, pid_lo + n_packages,
                       _ptr(tally), C.byref(st), _ptr(steps), _ptr(self_tally))
    stats = dict(escaped=st.escaped, capped=st.capped, steps=st.steps, emitted=st.emitted)
    return tally, stats, steps


def trace64(grid: Grid, *, source: int, kabs: float, ksca: float, g: float = 0.0,
            seed: int = 1, freq: int = 0, iteration: int = 0, cloud: int = 0,
            pid_lo: int = 0, n_packages: int, w0: int = W_UNIT, max_steps: int = 10_000_000,
            ps_pos=None, ps_cdf=None, n_per_cell: int = 1, leaf=None, dust_w=None,
            tally=None, want_steps: bool = False, dust_prefix=None):
    """The FP64 oracle on the same item and packages as :func:`trace` (same
    arguments; the opacities and g are taken as the same FP32 values).
    Returns (tally float64[n_cells] in weight units, stats dict with float
    escaped/emitted, per-package steps or None)."""
    if tally is None:
        tally = np.zeros(grid.n_cells, np.float64)
    ps_pos_a = None if ps_pos is None else np.ascontiguousarray(ps_pos, np.float32).ravel()
    ps_cdf_a = None if ps_cdf is None else np.ascontiguousarray(ps_cdf, np.float32)
    leaf_a = None if leaf is None else np.ascontiguousarray(leaf, np.int32)
    dust_a = None if dust_w is None else np.ascontiguousarray(dust_w, np.uint64)
    pref_a = None if dust_prefix is None else np.ascontiguousarray(dust_prefix, np.uint64)
    it = _Item(source, freq, iteration, cloud, seed & (2**64 - 1),
               np.float32(kabs), np.float32(ksca), np.float32(g), w0, max_steps,
               0 if ps_cdf_a is None else ps_cdf_a.size, _ptr(ps_pos_a), _ptr(ps_cdf_a),
               n_per_cell, 0 if leaf_a is None else leaf_a.size, _ptr(leaf_a), _ptr(dust_a), _ptr(pref_a))
    st = _Stats64()
    steps = np.zeros(n_packages, np.uint32) if want_steps else None
    gc = grid._c()
    lib64().oracle64_trace(C.byref(gc), C.byref(it), pid_lo, pid_lo + n_packages, _ptr(tally), C.byref(st),
                           _ptr(steps))
    stats = dict(escaped=st.escaped, capped=st.capped, steps=st.steps, emitted=st.emitted)
    return tally, stats, steps


def trace_pencil(grid: Grid, pos, direction, *, kabs: float, ksca: float = 0.0, g: float = 0.0,
                 seed: int = 1, pid: int = 0, w0: int = W_UNIT, max_steps: int = 10_000_000):
    """One package started at root-unit ``pos`` with ``direction`` (a pencil
    beam).  Returns (tally, stats, steps)."""
    tally = np.zeros(grid.n_cells, np.int64)
    it = _Item(SRC_POINT, 0, 0, 0, seed, np.float32(kabs), np.float32(ksca), np.float32(g),
               w0, max_steps, 0, None, None, 1, 0, None, None, None)
    st = _Stats()
    pos_a = np.ascontiguousarray(pos, np.float32)
    dir_a = np.ascontiguousarray(direction, np.float32)
    gc = grid._c()
    n = lib().oracle_trace_pencil(C.byref(gc), C.byref(it), _ptr(pos_a), _ptr(dir_a), pid,
                                  _ptr(tally), C.byref(st))
    stats = dict(escaped=st.escaped, capped=st.capped, steps=st.steps, emitted=st.emitted)
    return tally, stats, int(n)
