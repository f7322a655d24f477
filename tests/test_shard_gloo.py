"""Sharded tracing on two CPU ranks (gloo): each rank traces its package range
with the oracle, one int64 all-reduce sums the counters, and the result is
bit-identical to one process tracing every package.  The product's sharded
iteration (shard.iterate_sharded: iteration 0 and frozen-seed dust
iterations, every item's package ids split across the ranks, one counter
all-reduce per launch, A and T on every rank) is driven here with the oracle
as its backend and must give the one-rank temperatures bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1812_06632_gb300 import shard


def test_package_ranges():
    assert shard.package_range(0, 2, 10) == (0, 10)
    assert shard.package_range(1, 2, 10) == (10, 10)
    with pytest.raises(ValueError):
        shard.package_range(2, 2, 10)
    items = shard.shard_items([dict(source=0, freq=3, n_packages=7, pid_offset=5)], 1, 4)
    assert items[0]["pid_offset"] == 12 and items[0]["n_packages"] == 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from paper_1812_06632_gb300 import inputs as I, shard as S
    from parity_helpers import oracle_item
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.config_c2(n=10, n_freq=8, n_packages=0)
    specs = S.shard_items([dict(source=0, freq=f, n_packages=600) for f in (2, 6)], rank, world)
    tal = np.stack([oracle_item(w, 0, s)[0] for s in specs])
    t = torch.from_numpy(tal)
    S.allreduce_counters(t)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), t.numpy())
    dist.destroy_process_group()


def test_two_rank_allreduce_equals_single_process(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    from paper_1812_06632_gb300 import inputs as I
    from parity_helpers import oracle_item
    w = I.config_c2(n=10, n_freq=8, n_packages=0)
    ref = np.stack([oracle_item(w, 0, dict(source=0, freq=f, n_packages=1200))[0] for f in (2, 6)])
    for r in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"rank{r}.npy"), ref)


def test_split_range_covers_every_id_once():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard.split_range(n, r, world) for r in range(world)]
            ids = np.concatenate([np.arange(o, o + c) for o, c in parts])
            np.testing.assert_array_equal(ids, np.arange(n))
    with pytest.raises(ValueError):
        shard.split_range(2 ** 32 + 1, 0, 2)


class OracleBackend:
    """The oracle (FP32-contract tracer, FP64 physics) behind the five
    operations iterate_sharded needs; CPU torch tensors, so gloo can reduce
    the counters."""

    def __init__(self, w):
        import torch
        from oracle import physics as P
        from parity_helpers import oracle_grid
        self.w, self.P, self.torch = w, P, torch
        cl = w.clouds[0]
        self.cl = cl
        self.n_cells, self.n_freq = cl.n_cells, len(w.dust.nu)
        self.leaf = cl.leaves()
        self.n_leaf = self.leaf.size
        self.V = P.cell_volumes(oracle_grid(cl), cl.ell)

    def zeros(self, n, dtype):
        t = self.torch
        return t.zeros(n, dtype={"i8": t.int64, "f8": t.float64, "f4": t.float32}[dtype])

    def trace(self, specs, tally):
        from parity_helpers import oracle_item
        steps = 0
        for s in specs:
            s2 = {k: v for k, v in s.items() if k != "dust_w"}
            dw = None if s.get("dust_w") is None else s["dust_w"].numpy().astype(np.uint64)
            t, st, _ = oracle_item(self.w, 0, s2, dust_w=dw)
            o = s["tally_offset"]
            tally[o:o + self.n_cells] += self.torch.from_numpy(t.astype(np.int64))
            steps += int(st["steps"])
        return steps

    def package_energy(self, source, n_total):
        cl, P = self.cl, self.P
        if source == 0:
            return P.background_package_energy(self.w.bg_I[0], cl.nx, cl.ny, cl.nz, cl.ell, n_total)
        return P.point_package_energy(np.asarray(self.w.ps_L[0]).sum(axis=0), n_total)

    def absorbed_power(self, tally, e_unit, A_in, A_out):
        A = self.P.absorbed_power(tally.numpy().reshape(self.n_freq, self.n_cells), np.asarray(e_unit),
                                  self.w.dust.nu, self.cl.rho, self.V, A_in=A_in.numpy())
        A_out[:] = self.torch.from_numpy(A)

    def temperature(self, A, T):
        Tl = self.P.temperatures(A.numpy()[self.leaf], self.w.dust.nu, self.w.dust.kabs).astype(np.float32)
        old = T.numpy()[self.leaf]
        T[self.torch.from_numpy(self.leaf.astype(np.int64))] = self.torch.from_numpy(Tl)
        return float(np.abs(Tl.astype(np.float64) - old).max())

    def dust_emission(self, T, n_per_cell):
        P, w, lf = self.P, self.w, self.leaf
        W = np.zeros((self.n_freq, self.n_leaf), np.int64)
        e = np.zeros(self.n_freq)
        for f in range(self.n_freq):
            L = P.dust_luminosity(T.numpy()[lf].astype(np.float64), self.cl.rho[lf], self.V[lf], w.dust.kabs[f],
                                  w.dust.nu[f])
            Wd, e[f] = P.dust_weights(L, n_per_cell)
            W[f] = Wd.astype(np.int64)
        return self.torch.from_numpy(W), e

    def copy(self, dst, src):
        dst.copy_(src)


def _iter_workload():
    from paper_1812_06632_gb300 import inputs as I
    return I.config_c3(root_n=5, max_refine=1, sigma=1.5, threshold=2.0, tau_peak_1um=40.0, n_freq=6,
                       L_bol=3e36, side_pc=0.05)


ITER_KW = dict(n_background=301, n_point=257, n_per_cell=1, max_iter=2, dT_tol=0.0)


def _iter_worker(rank, world, port, out_dir):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from paper_1812_06632_gb300 import shard as S
    from test_shard_gloo import OracleBackend, _iter_workload, ITER_KW
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    be = OracleBackend(_iter_workload())
    T = torch.zeros(be.n_cells, dtype=torch.float32)
    r = S.iterate_sharded(be, T, rank=rank, world=world, **ITER_KW)
    np.save(os.path.join(out_dir, f"T{rank}.npy"), T.numpy())
    np.save(os.path.join(out_dir, f"steps{rank}.npy"), np.array([r["steps"], r["iterations"]]))
    dist.destroy_process_group()


def test_sharded_iteration_on_two_ranks_equals_one_rank(tmp_path):
    import torch
    world = 2
    mp.start_processes(_iter_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    be = OracleBackend(_iter_workload())
    T = torch.zeros(be.n_cells, dtype=torch.float32)
    r = shard.iterate_sharded(be, T, rank=0, world=1, **ITER_KW)
    assert r["iterations"] == 2 and T.max().item() > 10.0
    steps = 0
    for k in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"T{k}.npy"), T.numpy())
        s, it = np.load(tmp_path / f"steps{k}.npy")
        assert it == 2
        steps += int(s)
    assert steps == r["steps"]            # the ranks traced disjoint package ranges of the same items
