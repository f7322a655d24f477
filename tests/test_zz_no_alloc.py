"""The allocation-free tracer entry point (soc_simulate_frequency_batch_noalloc).

Callers that cannot allocate device memory mid-run -- code under a
framework's caching allocator or a fixed memory budget, real-time loops in
which cudaMalloc/cudaFree would synchronise the device -- use this variant; it
keeps its scratch in a fixed array inside the library.  Its counters must
equal those of the ordinary entry point exactly (integer fixed point), on two
calls in a row: the shared scratch keeps the previous call's contents, so the
second call also checks that the work counter is cleared.  The grid table is
exercised with two uploaded grids (a regular grid and an octree) whose items
alternate.  This file is collected last so that a failure here comes after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1812_06632_gb300 import inputs as I
from parity_helpers import gpu_context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _specs(cl, nl, dw):
    return [dict(source=0, freq=30, n_packages=5001, tally_offset=0),
            dict(source=1, freq=44, n_packages=3003, tally_offset=cl.n_cells),
            dict(source=0, freq=60, pid_offset=777, n_packages=2500, tally_offset=2 * cl.n_cells),
            dict(source=2, freq=12, n_packages=nl, n_per_cell=1, dust_w=dw, tally_offset=3 * cl.n_cells)]


def test_noalloc_entry_matches_ordinary_entry_twice(libsoc):
    w = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0, tau_peak_1um=30.0)
    cl = w.clouds[0]
    ctx, ids = gpu_context(w)
    nl = cl.leaves().size
    rng = np.random.default_rng(5)
    dw = torch.from_numpy(rng.integers(0, 2 ** 31, nl).astype(np.int64)).cuda()
    specs = _specs(cl, nl, dw)
    items = ctx.items(specs)
    total = sum(s["n_packages"] for s in specs)
    n = 4 * cl.n_cells

    def run(fn):
        tally = torch.zeros(n, dtype=torch.int64, device="cuda")
        stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
        steps = torch.zeros(total, dtype=torch.int32, device="cuda")
        st = fn(ctx.h, C.cast(items, C.c_void_p), len(items), C.c_void_p(tally.data_ptr()),
                C.c_void_p(stats.data_ptr()), C.c_void_p(steps.data_ptr()),
                C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, libsoc.lib.soc_last_error(ctx.h)
        torch.cuda.synchronize()
        return tally.cpu().numpy(), stats.cpu().numpy(), steps.cpu().numpy()

    ref = run(libsoc.lib.soc_simulate_frequency_batch)
    assert ref[1][:, 3].sum() > 0
    for _ in range(2):
        got = run(libsoc.lib.soc_simulate_frequency_batch_noalloc)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)


def _two_grid_workload():
    """An octree and a regular lognormal grid sharing one dust table."""
    wo = I.config_c3(root_n=8, max_refine=2, sigma=2.0, threshold=3.0, tau_peak_1um=30.0, n_freq=16)
    reg = I.regular(I.lognormal_density(16, 9, 1.5, -3.5).astype(np.float32) * np.float32(2.0),
                    ell=wo.clouds[0].ell)
    nu = wo.dust.nu
    return I.Workload("two_grids", [wo.clouds[0], reg], wo.dust, [wo.bg_I[0], I.diluted_blackbodies(nu)],
                      [wo.ps_pos[0], np.array([[8.0, 7.5, 9.0]])],
                      [wo.ps_L[0], wo.ps_L[0][:1]], [0, 0], [0, 0], seed=3)


def test_noalloc_two_grids_alternating_items_twice(libsoc):
    w = _two_grid_workload()
    ctx, ids = gpu_context(w)
    n0, n1 = w.clouds[0].n_cells, w.clouds[1].n_cells
    nl1 = w.clouds[1].leaves().size
    dw = torch.full((nl1,), 2 ** 30, dtype=torch.int64, device="cuda")
    specs = [dict(cloud=ids[0], source=0, freq=3, n_packages=3001, tally_offset=0),
             dict(cloud=ids[1], source=1, freq=5, n_packages=2002, tally_offset=n0),
             dict(cloud=ids[0], source=1, freq=9, n_packages=1500, tally_offset=n0 + n1),
             dict(cloud=ids[1], source=2, freq=11, n_packages=nl1, n_per_cell=1, dust_w=dw,
                  tally_offset=2 * n0 + n1),
             dict(cloud=ids[1], source=0, freq=14, pid_offset=99, n_packages=2500, tally_offset=2 * n0 + 2 * n1)]
    items = ctx.items(specs)
    total = sum(s["n_packages"] for s in specs)
    n = 2 * n0 + 3 * n1

    def run(fn):
        tally = torch.zeros(n, dtype=torch.int64, device="cuda")
        stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
        steps = torch.zeros(total, dtype=torch.int32, device="cuda")
        st = fn(ctx.h, C.cast(items, C.c_void_p), len(items), C.c_void_p(tally.data_ptr()),
                C.c_void_p(stats.data_ptr()), C.c_void_p(steps.data_ptr()),
                C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, libsoc.lib.soc_last_error(ctx.h)
        torch.cuda.synchronize()
        return tally.cpu().numpy(), stats.cpu().numpy(), steps.cpu().numpy()

    ref = run(libsoc.lib.soc_simulate_frequency_batch)
    assert (ref[1][:, 3] > 0).all()
    for _ in range(2):
        got = run(libsoc.lib.soc_simulate_frequency_batch_noalloc)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)


def test_noalloc_refuses_more_than_64_grids(libsoc):
    w = I.config_c1(n_packages=10)
    ctx, ids = gpu_context(w)
    small = I.regular(np.ones((2, 2, 2), np.float32))
    for _ in range(64):
        ctx.grid_upload(small)
    items = ctx.items([dict(source=0, freq=0, n_packages=10)])
    tally = torch.zeros(w.clouds[0].n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((1, 4), dtype=torch.int64, device="cuda")
    st = libsoc.lib.soc_simulate_frequency_batch_noalloc(
        ctx.h, C.cast(items, C.c_void_p), 1, C.c_void_p(tally.data_ptr()), C.c_void_p(stats.data_ptr()), None, None)
    assert st == -1
    assert b"64" in libsoc.lib.soc_last_error(ctx.h)


def test_direct_entries_refuse_a_capturing_stream(libsoc):
    """Both direct tracer entries copy tables from host memory: under stream
    capture they return SOC_ERR_STATE instead of recording a copy."""
    w = I.config_c1(n_packages=10)
    ctx, ids = gpu_context(w)
    items = ctx.items([dict(source=0, freq=0, n_packages=10)])
    tally = torch.zeros(w.clouds[0].n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((1, 4), dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g, stream=side):
        for fn in (libsoc.lib.soc_simulate_frequency_batch_noalloc, libsoc.lib.soc_simulate_frequency_batch):
            codes.append(fn(ctx.h, C.cast(items, C.c_void_p), 1, C.c_void_p(tally.data_ptr()),
                            C.c_void_p(stats.data_ptr()), None, C.c_void_p(side.cuda_stream)))
        tally.add_(1)
    g.replay()
    torch.cuda.synchronize()
    assert codes == [-5, -5]
    assert b"captured" in libsoc.lib.soc_last_error(ctx.h)
    assert int(tally.min()) == 1 and int(stats.abs().sum()) == 0
    # the context still works outside the capture
    ctx.simulate_noalloc(items, tally, stats)
    torch.cuda.synchronize()
    assert int(stats[0, 3]) == 10 * (1 << 31)


def test_noalloc_rejects_sizes_beyond_its_limit(libsoc):
    w = I.config_c1(n_packages=10)
    ctx, ids = gpu_context(w)
    too_many = ctx.items([dict(source=0, freq=0, n_packages=1)] * 1025)
    tally = torch.zeros(w.clouds[0].n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((1025, 4), dtype=torch.int64, device="cuda")
    st = libsoc.lib.soc_simulate_frequency_batch_noalloc(
        ctx.h, C.cast(too_many, C.c_void_p), 1025, C.c_void_p(tally.data_ptr()), C.c_void_p(stats.data_ptr()),
        None, None)
    assert st == -1
    assert b"1024" in libsoc.lib.soc_last_error(ctx.h)
