"""Sharded tracing on two CPU ranks (gloo): each rank traces its package range
with the oracle, one int64 all-reduce sums the counters, and the result is
bit-identical to one process tracing every package."""
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
