"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
CUDA library (through the C-ABI binding) and to the CPU oracle."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import physics as P

W_UNIT = 1 << 31


def oracle_grid(cl):
    return oracle.Grid(cl.nx, cl.ny, cl.nz, cl.level_start, cl.rho, cl.child, cl.parent)


def kappa_root(dust, f, ell):
    """FP32 opacity per root-cell length, as the library derives it."""
    return (np.float32(np.float64(dust.kabs[f]) * np.float64(ell)),
            np.float32(np.float64(dust.ksca[f]) * np.float64(ell)))


def oracle_item(w, ci, spec, dust_w=None, dust_prefix=None):
    """Run one batch item on the oracle; returns (tally, stats, steps)."""
    cl = w.clouds[ci]
    f = spec.get("freq", 0)
    ka, ks = kappa_root(w.dust, f, cl.ell)
    kw = dict(source=spec["source"], kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed, freq=f,
              iteration=spec.get("iteration", 0), cloud=ci, pid_lo=spec.get("pid_offset", 0),
              n_packages=spec["n_packages"], w0=spec.get("w0", W_UNIT), want_steps=True,
              max_steps=spec.get("max_steps", 10_000_000))
    if spec["source"] == oracle.SRC_POINT:
        kw["ps_pos"] = np.asarray(w.ps_pos[ci], np.float64).astype(np.float32)
        kw["ps_cdf"] = P.point_source_cdf(w.ps_L[ci])[f]
    if spec["source"] == oracle.SRC_DUST:
        kw["leaf"] = cl.leaves()
        kw["dust_w"] = dust_w
        kw["n_per_cell"] = spec.get("n_per_cell", 1)
        if dust_prefix is not None:
            kw["dust_prefix"] = dust_prefix
    return oracle.trace(oracle_grid(cl), **kw)


def gpu_context(w, seed=None, device=0):
    from paper_1812_06632_gb300 import soc
    ctx = soc.Context(device, w.seed if seed is None else seed)
    ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    ids = []
    for ci, cl in enumerate(w.clouds):
        cid = ctx.grid_upload(cl)
        ctx.sources_upload(cid, w.bg_I[ci], w.ps_pos[ci], w.ps_L[ci])
        ids.append(cid)
    return ctx, ids


def run_gpu(ctx, specs, tally_len, want_steps=True):
    """Run specs (dicts for Context.items) in one launch.  Returns numpy
    (tally, stats[n_items,4], pkg_steps)."""
    import torch
    items = ctx.items(specs)
    tally = torch.zeros(tally_len, dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    total = sum(s["n_packages"] for s in specs)
    steps = torch.zeros(max(total, 1), dtype=torch.int32, device="cuda") if want_steps else None
    ctx.simulate(items, tally, stats, steps)
    torch.cuda.synchronize()
    return (tally.cpu().numpy(), stats.cpu().numpy(),
            None if steps is None else steps.cpu().numpy().view(np.uint32)[:total])
