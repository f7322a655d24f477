"""ctypes binding of libsoc (include/soc.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts NumPy
arrays / torch tensors to pointers and raises on error statuses.  It raises
at import time if libsoc.so has not been built (there is no fallback).
Device buffers are torch CUDA tensors owned by the caller.

A run to converged temperatures, for a cloud built by ``inputs``::

    ctx = Context(0, seed=1)
    ctx.dust_upload(nu, kabs, ksca, g)              # FP64 tables per frequency
    cid = ctx.grid_upload(cloud)                    # validated, level-ordered octree
    ctx.sources_upload(cid, bg_I, ps_pos, ps_L)     # background and point sources
    T = torch.empty(cloud.n_cells, device="cuda")
    r = ctx.iterate(cid, T, n_background=10**6, n_point=10**6, max_iter=40, dT_tol=0.1)
    # r["iterations"], r["converged"], r["history"] (max |dT| per dust iteration)

Single tracer launches (``items`` / ``simulate``), prepared batches and CUDA
graphs, the FP64 normalisation and temperature steps, maps and the learned
seed are exposed one call each, as in the header.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SOC_LIB names another build of the same library (e.g. one compiled with
# different options); by default the in-tree build is loaded.
LIB_PATH = os.environ.get("SOC_LIB") or os.path.join(_HERE, "_build", "libsoc.so")

SOC_OK = 0
SOC_ERR_STEP_LIMIT = -4
SOC_ERR_STATE = -5
SOC_ERR_TIMEOUT = -7
SRC_BACKGROUND, SRC_POINT, SRC_DUST = 0, 1, 2
W_UNIT = 1 << 31

EXPORTS = ["soc_create", "soc_destroy", "soc_last_error", "soc_grid_upload", "soc_grid_validate", "soc_grid_free",
           "soc_dust_upload", "soc_simulate_frequency_batch_ex", "soc_update_temperature_ali", "soc_map",
           "soc_dust_weighted", "soc_dust_reweight", "soc_dust_luminosity", "soc_reference_delta",
           "soc_dust_split", "soc_reference_update",
           "soc_sources_upload", "soc_simulate_frequency_batch", "soc_package_energy",
           "soc_dust_emission", "soc_absorbed_power", "soc_update_temperature", "soc_iterate",
           "soc_set_launch", "soc_set_refill", "soc_set_scatter_batch", "soc_set_max_steps", "soc_probe_read",
           "soc_batch_create", "soc_batch_launch", "soc_batch_destroy", "soc_capture_begin",
           "soc_capture_end", "soc_graph_launch", "soc_graph_destroy",
           "soc_unet_create", "soc_unet_destroy", "soc_unet_param_count", "soc_unet_set_params",
           "soc_unet_get_params", "soc_unet_forward", "soc_unet_backward", "soc_unet_adam",
           "soc_nn_conv3d", "soc_nn_conv3d_dgrad", "soc_nn_conv3d_wgrad", "soc_nn_error_flag",
           "soc_simulate_frequency_batch_noalloc", "soc_abort", "soc_abort_clear", "soc_abort_status",
           "soc_set_timeout", "soc_nn_adam", "soc_seed_features", "soc_seed_transform",
           "soc_iterate_batch", "soc_nn_seed_features", "soc_nn_scale_add"]


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_levels", C.c_int32),
                ("cells_per_level", C.c_void_p), ("rho", C.c_void_p), ("first_child", C.c_void_p),
                ("parent", C.c_void_p), ("root_cell_size", C.c_double)]


class BatchItem(C.Structure):
    _fields_ = [("cloud", C.c_int32), ("freq", C.c_int32), ("source", C.c_int32),
                ("iteration", C.c_int32), ("pid_offset", C.c_uint64), ("n_packages", C.c_uint64),
                ("w0", C.c_uint64), ("tally_offset", C.c_int64), ("d_dust_w", C.c_void_p),
                ("n_per_cell", C.c_uint32), ("reserved", C.c_uint32)]


class IterateParams(C.Structure):
    _fields_ = [("n_background", C.c_uint64), ("n_point", C.c_uint64), ("n_per_cell", C.c_uint32),
                ("max_iter", C.c_int32), ("dT_tol", C.c_double), ("reuse_constant", C.c_int32),
                ("ali", C.c_int32), ("n_weighted", C.c_uint64), ("weighted_cap", C.c_uint32),
                ("reference_field", C.c_int32), ("n_dust_first", C.c_uint64), ("n_dust_last", C.c_uint64)]


SEED_MAX_BINS = 64


class SeedMap(C.Structure):
    _fields_ = [("y_mean", C.c_double), ("y_std", C.c_double), ("shrink", C.c_double), ("n_bins", C.c_int32),
                ("reserved", C.c_int32), ("lnT1_lo", C.c_double), ("lnT1_hi", C.c_double),
                ("y_lo", C.c_double * SEED_MAX_BINS), ("y_hi", C.c_double * SEED_MAX_BINS)]


def seed_map(y_mean, y_std, shrink=1.0, envelope=None):
    """SeedMap from the de-normalisation, the shrink factor and an optional
    envelope (lnT1_lo, lnT1_hi, y_lo[n], y_hi[n])."""
    m = SeedMap()
    m.y_mean, m.y_std, m.shrink = float(y_mean), float(y_std), float(shrink)
    if envelope is not None:
        lo, hi, ylo, yhi = envelope
        m.n_bins = len(ylo)
        m.lnT1_lo, m.lnT1_hi = float(lo), float(hi)
        for b in range(m.n_bins):
            m.y_lo[b], m.y_hi[b] = float(ylo[b]), float(yhi[b])
    return m


class IterateResult(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("final_max_dT", C.c_double),
                ("steps", C.c_int64), ("capped", C.c_int64)]


class SocError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsoc status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1812_06632_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    P, I, U64, D = C.c_void_p, C.c_int, C.c_uint64, C.c_double
    sig = {
        "soc_create": ([C.POINTER(P), I, U64], I),
        "soc_destroy": ([P], None),
        "soc_last_error": ([P], C.c_char_p),
        "soc_grid_upload": ([P, C.POINTER(GridDesc), C.POINTER(I)], I),
        "soc_grid_validate": ([C.POINTER(GridDesc), C.c_char_p, I], I),
        "soc_grid_free": ([P, I], I),
        "soc_dust_upload": ([P, I, P, P, P, P], I),
        "soc_sources_upload": ([P, I, P, I, P, P], I),
        "soc_simulate_frequency_batch": ([P, P, I, P, P, P, P], I),
        "soc_simulate_frequency_batch_ex": ([P, P, I, P, P, P, P, P], I),
        "soc_update_temperature_ali": ([P, I, P, P, P, P, P], I),
        "soc_map": ([P, I, P, I, P, P, I, I, C.c_double, P, C.c_double, P, P], I),
        "soc_dust_weighted": ([P, I, P, P, I, C.c_uint64, C.c_uint32, P, P, P], I),
        "soc_dust_reweight": ([P, I, P, P, I, P, P, P], I),
        "soc_dust_luminosity": ([P, I, P, I, I, P, P], I),
        "soc_reference_delta": ([P, I, I, P, P, C.c_double, P, P, P, P], I),
        "soc_dust_split": ([P, I, I, P, P, P, P, P, P], I),
        "soc_reference_update": ([P, I, P, P, C.c_double, P, P, I, P], I),
        "soc_package_energy": ([P, I, I, U64, P], I),
        "soc_dust_emission": ([P, I, P, I, I, C.c_uint32, P, P, P], I),
        "soc_absorbed_power": ([P, I, P, C.c_int64, P, P, P, P], I),
        "soc_update_temperature": ([P, I, P, P, P, P], I),
        "soc_iterate": ([P, I, C.POINTER(IterateParams), P, P, C.POINTER(IterateResult), P, P], I),
        "soc_set_launch": ([P, I, I, I], I),
        "soc_set_refill": ([P, I], I),
        "soc_set_scatter_batch": ([P, I], I),
        "soc_batch_create": ([P, P, I, C.POINTER(I)], I),
        "soc_batch_launch": ([P, I, P, C.c_int64, P, P, P], I),
        "soc_batch_destroy": ([P, I], I),
        "soc_capture_begin": ([P, P], I),
        "soc_capture_end": ([P, P, C.POINTER(I)], I),
        "soc_graph_launch": ([P, I, P], I),
        "soc_graph_destroy": ([P, I], I),
        "soc_unet_create": ([I, I, I, I, C.POINTER(I)], I),
        "soc_unet_destroy": ([I], I),
        "soc_unet_param_count": ([], C.c_int64),
        "soc_unet_set_params": ([I, P], I),
        "soc_unet_get_params": ([I, P, I], I),
        "soc_unet_forward": ([I, P, P, P], I),
        "soc_unet_backward": ([I, P, P, P, P, P], I),
        "soc_unet_adam": ([I, C.c_float, P], I),
        "soc_nn_conv3d": ([P, I, I, I, I, I, P, P, I, I, P, P, P], I),
        "soc_nn_error_flag": ([C.POINTER(I)], I),
        "soc_nn_conv3d_dgrad": ([P, I, I, I, I, I, P, I, P, P, P], I),
        "soc_nn_conv3d_wgrad": ([P, P, I, I, I, I, I, I, P, P, P], I),
        "soc_set_max_steps": ([P, C.c_uint32], I),
        "soc_probe_read": ([P, P, C.c_uint64, C.c_int32, P], I),
        "soc_simulate_frequency_batch_noalloc": ([P, P, I, P, P, P, P], I),
        "soc_abort": ([P], I),
        "soc_abort_clear": ([P], I),
        "soc_abort_status": ([P, C.POINTER(I), C.POINTER(I)], I),
        "soc_set_timeout": ([P, C.c_double], I),
        "soc_nn_adam": ([P, P, P, P, C.c_int64, C.c_float, C.c_int32, P, P], I),
        "soc_nn_scale_add": ([P, P, C.c_int64, C.c_float, P], I),
        "soc_seed_features": ([P, I, P, P, P, P, I, P, P], I),
        "soc_seed_transform": ([P, I, P, P, C.POINTER(SeedMap), P, P], I),
        "soc_iterate_batch": ([P, I, P, C.POINTER(IterateParams), P, P, P, P, P], I),
        "soc_nn_seed_features": ([P, P, P, P, C.c_int64, P, I, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _np_ptr(a):
    return None if a is None else a.ctypes.data


def _t_ptr(t):
    """Device pointer of a torch tensor.  Every tensor the library takes is
    caller-owned device memory read or written as one dense array: a host
    tensor or a strided view would have the kernels address the wrong memory,
    so both are refused here, before any launch."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsoc takes CUDA tensors (got a host tensor)")
    if not t.is_contiguous():
        raise ValueError("libsoc takes contiguous tensors (got a strided view)")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def grid_desc(nx, ny, nz, cells_per_level, rho, first_child=None, parent=None, ell=1.0):
    """GridDesc plus the arrays it points into (keep them alive together)."""
    keep = [np.ascontiguousarray(cells_per_level, np.int64), np.ascontiguousarray(rho, np.float32),
            None if first_child is None else np.ascontiguousarray(first_child, np.int32),
            None if parent is None else np.ascontiguousarray(parent, np.int32)]
    d = GridDesc(nx, ny, nz, keep[0].size, _np_ptr(keep[0]), _np_ptr(keep[1]), _np_ptr(keep[2]),
                 _np_ptr(keep[3]), float(ell))
    return d, keep


def validate_grid(nx, ny, nz, cells_per_level, rho, first_child=None, parent=None, ell=1.0):
    """soc_grid_validate: (status, message); host only, no GPU needed."""
    d, keep = grid_desc(nx, ny, nz, cells_per_level, rho, first_child, parent, ell)
    buf = C.create_string_buffer(512)
    st = lib.soc_grid_validate(C.byref(d), buf, 512)
    return st, buf.value.decode()


class Context:
    """One libsoc context (device + seed).  Methods mirror the C-ABI."""

    def __init__(self, device: int = 0, seed: int = 1):
        h = C.c_void_p()
        st = lib.soc_create(C.byref(h), device, seed & (2 ** 64 - 1))
        if st != SOC_OK:
            raise SocError(st, "soc_create failed (no CUDA device?)")
        self.h = h
        self.device = device
        self.n_freq = 0
        self.clouds = []

    def close(self):
        if self.h:
            lib.soc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, ok=(SOC_OK,)):
        if st not in ok:
            raise SocError(st, lib.soc_last_error(self.h).decode())
        return st

    # -- uploads ------------------------------------------------------------
    def grid_upload(self, cloud, *, paper_encoding: bool = False) -> int:
        """Upload an inputs.Cloud.  With paper_encoding the links travel as
        negative densities (the paper's format) instead of a child array."""
        cpl = np.ascontiguousarray(cloud.cells_per_level(), np.int64)
        if paper_encoding:
            rho = np.ascontiguousarray(cloud.paper_encoding(), np.float32)
            child = None
        else:
            rho = np.ascontiguousarray(cloud.rho, np.float32)
            child = np.ascontiguousarray(cloud.child, np.int32)
        parent = np.ascontiguousarray(cloud.parent, np.int32) if cloud.parent.size else None
        d = GridDesc(cloud.nx, cloud.ny, cloud.nz, cloud.n_levels, _np_ptr(cpl), _np_ptr(rho),
                     _np_ptr(child), _np_ptr(parent), float(cloud.ell))
        cid = C.c_int(-1)
        self._check(lib.soc_grid_upload(self.h, C.byref(d), C.byref(cid)))
        self.clouds.append(cloud)
        return cid.value

    def grid_upload_raw(self, nx, ny, nz, cells_per_level, rho, first_child=None, parent=None, ell=1.0) -> int:
        cpl = np.ascontiguousarray(cells_per_level, np.int64)
        rho = np.ascontiguousarray(rho, np.float32)
        fc = None if first_child is None else np.ascontiguousarray(first_child, np.int32)
        pa = None if parent is None else np.ascontiguousarray(parent, np.int32)
        d = GridDesc(nx, ny, nz, cpl.size, _np_ptr(cpl), _np_ptr(rho), _np_ptr(fc), _np_ptr(pa), float(ell))
        cid = C.c_int(-1)
        self._check(lib.soc_grid_upload(self.h, C.byref(d), C.byref(cid)))
        return cid.value

    def grid_free(self, cloud_id):
        self._check(lib.soc_grid_free(self.h, cloud_id))

    def dust_upload(self, nu, kabs, ksca, g):
        nu, kabs, ksca, g = (np.ascontiguousarray(a, np.float64) for a in (nu, kabs, ksca, g))
        self._check(lib.soc_dust_upload(self.h, nu.size, _np_ptr(nu), _np_ptr(kabs), _np_ptr(ksca), _np_ptr(g)))
        self.n_freq = nu.size

    def sources_upload(self, cloud_id, bg_I=None, ps_pos=None, ps_L=None):
        bg = None if bg_I is None else np.ascontiguousarray(bg_I, np.float64)
        n_ps = 0 if ps_pos is None else int(np.asarray(ps_pos).shape[0])
        pos = None if ps_pos is None else np.ascontiguousarray(ps_pos, np.float64).ravel()
        L = None if ps_L is None else np.ascontiguousarray(ps_L, np.float64).ravel()
        self._check(lib.soc_sources_upload(self.h, cloud_id, _np_ptr(bg), n_ps, _np_ptr(pos), _np_ptr(L)))

    def set_launch(self, threads_per_block=256, blocks_per_sm=0, chunk=1):
        self._check(lib.soc_set_launch(self.h, threads_per_block, blocks_per_sm, chunk))

    def set_refill(self, min_idle_lanes):
        self._check(lib.soc_set_refill(self.h, min_idle_lanes))

    def set_scatter_batch(self, min_lanes):
        self._check(lib.soc_set_scatter_batch(self.h, min_lanes))

    def set_max_steps(self, n):
        self._check(lib.soc_set_max_steps(self.h, n))

    def abort(self):
        """soc_abort: tracer launches of this context take no more work."""
        self._check(lib.soc_abort(self.h))

    def abort_clear(self):
        self._check(lib.soc_abort_clear(self.h))

    def abort_status(self):
        """(requested, cut): the abort flag, and whether a launch since the
        last clear left work untraced."""
        r, c = C.c_int(0), C.c_int(0)
        self._check(lib.soc_abort_status(self.h, C.byref(r), C.byref(c)))
        return bool(r.value), bool(c.value)

    def set_timeout(self, seconds: float):
        """soc_set_timeout: watchdog deadline of each iterate call (0 = none)."""
        self._check(lib.soc_set_timeout(self.h, float(seconds)))

    def probe_read(self, buf, reps: int, stream=None):
        """soc_probe_read: `reps` reads of the device tensor `buf` in one
        launch (measurement helper; the caller times it)."""
        self._check(lib.soc_probe_read(self.h, C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                       reps, _stream(stream)))

    # -- compute ------------------------------------------------------------
    @staticmethod
    def items(specs):
        """Array of BatchItem from dicts (keys as in soc_batch_item)."""
        arr = (BatchItem * len(specs))()
        for i, s in enumerate(specs):
            it = arr[i]
            it.cloud = s.get("cloud", 0)
            it.freq = s.get("freq", 0)
            it.source = s["source"]
            it.iteration = s.get("iteration", 0)
            it.pid_offset = s.get("pid_offset", 0)
            it.n_packages = s["n_packages"]
            it.w0 = s.get("w0", W_UNIT)
            it.tally_offset = s.get("tally_offset", 0)
            dw = s.get("dust_w")
            it.d_dust_w = None if dw is None else dw.data_ptr()
            it.n_per_cell = s.get("n_per_cell", 1)
            it.reserved = 1 if s.get("weighted") else 0
        return arr

    def simulate(self, items, tally, stats, pkg_steps=None, stream=None, self_tally=None):
        """soc_simulate_frequency_batch(_ex); items from Context.items()."""
        if self_tally is not None:
            return self._check(lib.soc_simulate_frequency_batch_ex(
                self.h, C.cast(items, C.c_void_p), len(items), _t_ptr(tally), _t_ptr(self_tally), _t_ptr(stats),
                _t_ptr(pkg_steps), _stream(stream)))
        return self._check(lib.soc_simulate_frequency_batch(
            self.h, C.cast(items, C.c_void_p), len(items), _t_ptr(tally), _t_ptr(stats),
            _t_ptr(pkg_steps), _stream(stream)))

    def simulate_noalloc(self, items, tally, stats, pkg_steps=None, stream=None):
        """soc_simulate_frequency_batch_noalloc: same results, no device
        allocation (fixed library-internal scratch; see include/soc.h)."""
        return self._check(lib.soc_simulate_frequency_batch_noalloc(
            self.h, C.cast(items, C.c_void_p), len(items), _t_ptr(tally), _t_ptr(stats),
            _t_ptr(pkg_steps), _stream(stream)))

    # -- prepared batches and CUDA graphs ----------------------------------
    def batch_create(self, items) -> int:
        bid = C.c_int(-1)
        self._check(lib.soc_batch_create(self.h, C.cast(items, C.c_void_p), len(items), C.byref(bid)))
        return bid.value

    def batch_launch(self, batch_id, tally, stats, pkg_steps=None, zero_tally=True, stream=None):
        self._check(lib.soc_batch_launch(self.h, batch_id, _t_ptr(tally), tally.numel() if zero_tally else 0,
                                         _t_ptr(stats), _t_ptr(pkg_steps), _stream(stream)))

    def batch_destroy(self, batch_id):
        self._check(lib.soc_batch_destroy(self.h, batch_id))

    def capture_begin(self, stream):
        self._check(lib.soc_capture_begin(self.h, _stream(stream)))

    def capture_end(self, stream) -> int:
        gid = C.c_int(-1)
        self._check(lib.soc_capture_end(self.h, _stream(stream), C.byref(gid)))
        return gid.value

    def graph_launch(self, graph_id, stream=None):
        self._check(lib.soc_graph_launch(self.h, graph_id, _stream(stream)))

    def graph_destroy(self, graph_id):
        self._check(lib.soc_graph_destroy(self.h, graph_id))

    def package_energy(self, cloud_id, source, n_packages):
        e = np.zeros(self.n_freq, np.float64)
        self._check(lib.soc_package_energy(self.h, cloud_id, source, n_packages, _np_ptr(e)))
        return e

    def dust_emission(self, cloud_id, T, w, e_unit, n_per_cell=1, freq_lo=0, n_freq=None, stream=None):
        n_freq = self.n_freq - freq_lo if n_freq is None else n_freq
        self._check(lib.soc_dust_emission(self.h, cloud_id, _t_ptr(T), freq_lo, n_freq, n_per_cell,
                                          _t_ptr(w), _t_ptr(e_unit), _stream(stream)))

    def dust_weighted(self, cloud_id, u, e_unit_uniform, n_total, cap, out, e_unit, stream=None):
        """soc_dust_weighted: out = [n_freq][2 n_leaf + 1] (weights, prefix)."""
        n_freq = u.shape[0]
        self._check(lib.soc_dust_weighted(self.h, cloud_id, _t_ptr(u), _t_ptr(e_unit_uniform), n_freq, n_total, cap,
                                          _t_ptr(out), _t_ptr(e_unit), _stream(stream)))

    def dust_reweight(self, cloud_id, u, e_unit_uniform, inout, e_unit, stream=None):
        """soc_dust_reweight: new weights for the allocation held in inout."""
        self._check(lib.soc_dust_reweight(self.h, cloud_id, _t_ptr(u), _t_ptr(e_unit_uniform), u.shape[0],
                                          _t_ptr(inout), _t_ptr(e_unit), _stream(stream)))

    def dust_luminosity(self, cloud_id, T, L, freq_lo=0, stream=None):
        """soc_dust_luminosity: L (float64 [n_freq][n_leaf]) from T."""
        self._check(lib.soc_dust_luminosity(self.h, cloud_id, _t_ptr(T), freq_lo, L.shape[0], _t_ptr(L),
                                            _stream(stream)))

    def reference_delta(self, cloud_id, L, L_ref, w, u, neg, e_unit_uniform, stream=None):
        """soc_reference_delta: u (int64 view of uint64), neg (uint8), e; L_ref updated."""
        self._check(lib.soc_reference_delta(self.h, cloud_id, L.shape[0], _t_ptr(L), _t_ptr(L_ref), float(w),
                                            _t_ptr(u), _t_ptr(neg), _t_ptr(e_unit_uniform), _stream(stream)))

    def dust_split(self, cloud_id, neg, alloc, alloc_neg, e_unit, e_unit_neg, stream=None):
        self._check(lib.soc_dust_split(self.h, cloud_id, alloc.shape[0], _t_ptr(neg), _t_ptr(alloc),
                                       _t_ptr(alloc_neg), _t_ptr(e_unit), _t_ptr(e_unit_neg), _stream(stream)))

    def reference_update(self, cloud_id, A_ref, A_d, w, A_const=None, A_out=None, out_mean=False, stream=None):
        self._check(lib.soc_reference_update(self.h, cloud_id, _t_ptr(A_ref), _t_ptr(A_d), float(w),
                                             _t_ptr(A_const), _t_ptr(A_out), int(out_mean), _stream(stream)))

    def absorbed_power(self, cloud_id, tally, stride, e_unit, A_out, A_in=None, stream=None):
        self._check(lib.soc_absorbed_power(self.h, cloud_id, _t_ptr(tally), stride, _t_ptr(e_unit),
                                           _t_ptr(A_in), _t_ptr(A_out), _stream(stream)))

    def map(self, cloud_id, T, freq, direction, up, npx, npy, pix_size, center, out, I_bg=0.0, stream=None):
        """soc_map: surface-brightness map into out (torch float32 [npy, npx])."""
        d = np.ascontiguousarray(direction, np.float64)
        u = np.ascontiguousarray(up, np.float64)
        c = np.ascontiguousarray(center, np.float64)
        self._check(lib.soc_map(self.h, cloud_id, _t_ptr(T), freq, _np_ptr(d), _np_ptr(u), npx, npy,
                                float(pix_size), _np_ptr(c), float(I_bg), _t_ptr(out), _stream(stream)))

    def seed_features(self, cloud_id, T, norm, x, T_prev=None, T_prev2=None, stream=None):
        """soc_seed_features: x (float32 [n_cells, n_features]) from T, the
        grid's density, (3 or 4 features) T_prev and (4 features) T_prev2;
        norm = {mean, width} of each feature (4, 6 or 8 values)."""
        nrm = np.ascontiguousarray(norm, np.float64)
        self._check(lib.soc_seed_features(self.h, cloud_id, _t_ptr(T), _t_ptr(T_prev), _t_ptr(T_prev2), _np_ptr(nrm),
                                          nrm.size // 2, _t_ptr(x), _stream(stream)))

    def seed_transform(self, cloud_id, T1, pred, smap, T_seed, stream=None):
        """soc_seed_transform: T_seed = clamp(T1 exp(y)) with y the
        de-normalised, shrunk and envelope-bounded prediction (smap: SeedMap,
        see seed_map)."""
        self._check(lib.soc_seed_transform(self.h, cloud_id, _t_ptr(T1), _t_ptr(pred), C.byref(smap), _t_ptr(T_seed),
                                           _stream(stream)))

    def update_temperature_ali(self, cloud_id, A, A_self, T, max_dT=None, stream=None):
        self._check(lib.soc_update_temperature_ali(self.h, cloud_id, _t_ptr(A), _t_ptr(A_self), _t_ptr(T),
                                                   _t_ptr(max_dT), _stream(stream)))

    def update_temperature(self, cloud_id, A, T, max_dT=None, stream=None):
        self._check(lib.soc_update_temperature(self.h, cloud_id, _t_ptr(A), _t_ptr(T), _t_ptr(max_dT),
                                               _stream(stream)))

    def iterate(self, cloud_id, T_out, *, n_background=0, n_point=0, n_per_cell=1, max_iter=0,
                dT_tol=0.1, T_seed=None, reuse_constant=False, ali=False, n_weighted=0, weighted_cap=10000,
                reference_field=False, n_dust_first=0, n_dust_last=0, stream=None):
        """soc_iterate: the iteration driver.  Iteration 0 traces the constant
        sources (n_background / n_point packages per frequency) and solves T;
        each dust iteration re-emits from the previous T (n_per_cell per leaf,
        or n_weighted in all with at most weighted_cap per cell) with frozen
        random numbers, until max |dT| < dT_tol or max_iter.  T_seed (device
        float [n_cells]) replaces the constant sources' T as the dust start;
        reuse_constant=True skips iteration 0 and reuses the constant-source
        absorption of the previous call on this cloud; ali=True uses the
        diagonal operator; reference_field "mean" or
        "difference" with package counts growing from n_dust_first to
        n_dust_last.  T_out receives the temperatures.  Returns iterations,
        converged, final_max_dT, steps, capped, the max |dT| history and
        timed_out (the abort flag or the set_timeout deadline stopped it)."""
        modes = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, "mean": 1, "difference": 2}
        p = IterateParams(n_background, n_point, n_per_cell, max_iter, dT_tol, int(reuse_constant), int(ali),
                          n_weighted, weighted_cap, modes[reference_field], n_dust_first, n_dust_last)
        r = IterateResult()
        hist = np.zeros(max(max_iter, 1), np.float64)
        st = self._check(lib.soc_iterate(self.h, cloud_id, C.byref(p), _t_ptr(T_seed), _t_ptr(T_out), C.byref(r),
                                         _np_ptr(hist), _stream(stream)),
                         ok=(SOC_OK, SOC_ERR_STEP_LIMIT, SOC_ERR_TIMEOUT))
        return dict(iterations=r.iterations, converged=bool(r.converged), final_max_dT=r.final_max_dT,
                    steps=r.steps, capped=r.capped, history=hist[:r.iterations].copy(),
                    timed_out=st == SOC_ERR_TIMEOUT)

    def iterate_batch(self, cloud_ids, T_outs, *, n_background=0, n_point=0, n_per_cell=1, max_iter=0, dT_tol=0.1,
                       T_seeds=None, reuse_constant=False, ali=False, stream=None):
        """soc_iterate_batch: soc_iterate for several clouds, one tracer launch per
        iteration for all clouds not yet converged.  T_outs / T_seeds: lists of
        device tensors (T_seeds entries may be None).  Returns one dict per cloud
        (as iterate) and timed_out."""
        n = len(cloud_ids)
        ids = (C.c_int * n)(*cloud_ids)
        outs = (C.c_void_p * n)(*[t.data_ptr() for t in T_outs])
        for t in T_outs:
            _t_ptr(t)
        seeds = None
        if T_seeds is not None:
            seeds = (C.c_void_p * n)(*[None if t is None else _t_ptr(t).value for t in T_seeds])
        p = IterateParams(n_background, n_point, n_per_cell, max_iter, dT_tol, int(reuse_constant), int(ali), 0, 0, 0, 0, 0)
        res = (IterateResult * n)()
        hist = np.zeros((n, max(max_iter, 1)), np.float64)
        st = self._check(lib.soc_iterate_batch(self.h, n, ids, C.byref(p), seeds, outs, res, _np_ptr(hist),
                                               _stream(stream)), ok=(SOC_OK, SOC_ERR_STEP_LIMIT, SOC_ERR_TIMEOUT))
        rows = [dict(iterations=r.iterations, converged=bool(r.converged), final_max_dT=r.final_max_dT, steps=r.steps,
                     capped=r.capped, history=hist[k, :r.iterations].copy()) for k, r in enumerate(res)]
        return rows, st == SOC_ERR_TIMEOUT


def _nn_check(st, what):
    if st != SOC_OK:
        raise SocError(st, what)


class UNet:
    """The learned temperature seed (soc_unet_*): 3D U-Net on cubes of side
    `side` (multiple of 8), batch `batch`; input (N,S,S,S,n_inputs) FP32,
    output (N,S,S,S) FP32, all torch CUDA tensors."""

    def __init__(self, batch: int, side: int, device: int = 0, n_inputs: int = 2):
        nid = C.c_int(-1)
        _nn_check(lib.soc_unet_create(device, batch, side, n_inputs, C.byref(nid)), "soc_unet_create")
        self.id = nid.value
        self.batch, self.side, self.n_inputs = batch, side, n_inputs
        self.n_params = int(lib.soc_unet_param_count())

    def close(self):
        if self.id is not None:
            lib.soc_unet_destroy(self.id)
            self.id = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.n_params
        _nn_check(lib.soc_unet_set_params(self.id, _np_ptr(flat)), "soc_unet_set_params")

    def get_params(self, grads: bool = False):
        out = np.empty(self.n_params, np.float32)
        _nn_check(lib.soc_unet_get_params(self.id, _np_ptr(out), int(grads)), "soc_unet_get_params")
        return out

    def forward(self, x, pred, stream=None):
        _nn_check(lib.soc_unet_forward(self.id, _t_ptr(x), _t_ptr(pred), _stream(stream)), "soc_unet_forward")

    def backward(self, x, target, pred=None, loss=None, stream=None):
        _nn_check(lib.soc_unet_backward(self.id, _t_ptr(x), _t_ptr(target), _t_ptr(pred), _t_ptr(loss),
                                        _stream(stream)), "soc_unet_backward")

    def adam(self, lr, stream=None):
        _nn_check(lib.soc_unet_adam(self.id, C.c_float(lr), _stream(stream)), "soc_unet_adam")


def nn_error_flag():
    """soc_nn_error_flag: 1 if a tensor-core convolution block timed out
    (the flag is cleared)."""
    f = C.c_int(0)
    _nn_check(lib.soc_nn_error_flag(C.byref(f)), "soc_nn_error_flag")
    return f.value


def conv3d(x, w, bias=None, relu=False, out=None, out_f32=None, stream=None):
    """soc_nn_conv3d on channels-last BF16 tensors (N, D, H, W, C)."""
    N, D, H, W, Cin = x.shape
    Cout = w.shape[0]
    _nn_check(lib.soc_nn_conv3d(_t_ptr(x), N, D, H, W, Cin, _t_ptr(w), _t_ptr(bias), Cout, int(relu),
                                _t_ptr(out), _t_ptr(out_f32), _stream(stream)), "soc_nn_conv3d")


def conv3d_dgrad(gy, w, w_scratch, gx, stream=None):
    N, D, H, W, Cout = gy.shape
    Cin = w.shape[2]
    _nn_check(lib.soc_nn_conv3d_dgrad(_t_ptr(gy), N, D, H, W, Cout, _t_ptr(w), Cin, _t_ptr(w_scratch),
                                      _t_ptr(gx), _stream(stream)), "soc_nn_conv3d_dgrad")


def seed_features(T, rho, norm, x, T_prev=None, T_prev2=None, stream=None):
    """soc_nn_seed_features: x (float32 [n, n_features]) from device T, rho,
    (3 or 4 features) T_prev and (4 features) T_prev2; norm = {mean, width}
    of each feature."""
    nrm = np.ascontiguousarray(norm, np.float64)
    _nn_check(lib.soc_nn_seed_features(_t_ptr(T), _t_ptr(T_prev), _t_ptr(T_prev2), _t_ptr(rho), T.numel(),
                                       _np_ptr(nrm), nrm.size // 2, _t_ptr(x), _stream(stream)), "soc_nn_seed_features")


def scale_add(y, x, a, stream=None):
    """soc_nn_scale_add: y <- fma(a, x, y) on FP32 device tensors of one size."""
    if y.numel() != x.numel():
        raise ValueError("y and x differ in size")
    _nn_check(lib.soc_nn_scale_add(_t_ptr(y), _t_ptr(x), y.numel(), C.c_float(a), _stream(stream)),
              "soc_nn_scale_add")


def adam(w, m, v, g, lr, t, w_bf16=None, stream=None):
    """soc_nn_adam: one Adam step at step t on FP32 device tensors."""
    _nn_check(lib.soc_nn_adam(_t_ptr(w), _t_ptr(m), _t_ptr(v), _t_ptr(g), w.numel(), C.c_float(lr), int(t),
                              _t_ptr(w_bf16), _stream(stream)), "soc_nn_adam")


def conv3d_wgrad(gy, x, gw, gb=None, stream=None):
    N, D, H, W, Cout = gy.shape
    Cin = x.shape[4]
    _nn_check(lib.soc_nn_conv3d_wgrad(_t_ptr(gy), _t_ptr(x), N, D, H, W, Cin, Cout, _t_ptr(gw), _t_ptr(gb),
                                      _stream(stream)), "soc_nn_conv3d_wgrad")
