"""Host logic of the autotuner (no GPU): candidate space, keys, cache."""
import numpy as np

from paper_1812_06632_gb300 import autotune as A
from paper_1812_06632_gb300 import inputs as I


def test_candidates_cover_space():
    c = list(A.candidates(dict(threads_per_block=(64, 128), blocks_per_sm=(0,), chunk=(1, 4), refill=(1,),
                               scatter=(1, 8))))
    assert len(c) == 8
    assert {x["threads_per_block"] for x in c} == {64, 128}
    assert {x["scatter"] for x in c} == {1, 8}
    assert len(list(A.candidates())) == 2 * 2 * 2 * 3 * 4


def test_key_depends_on_workload_and_gpu():
    cl = [I.regular(np.ones((4, 4, 4), np.float32))]
    s1 = [dict(source=0, freq=0, n_packages=10)]
    s2 = [dict(source=0, freq=0, n_packages=11)]
    assert A.workload_key("g", s1, cl) == A.workload_key("g", s1, cl)
    assert A.workload_key("g", s1, cl) != A.workload_key("g", s2, cl)
    assert A.workload_key("g", s1, cl) != A.workload_key("h", s1, cl)


def test_cache_roundtrip_and_pick(tmp_path):
    p = str(tmp_path / "c.json")
    assert A.load_cache(p) == {}
    res = [(dict(threads_per_block=128, blocks_per_sm=0, chunk=1, refill=1), 3.0),
           (dict(threads_per_block=256, blocks_per_sm=4, chunk=4, refill=8), 2.0)]
    best = A.pick(res)
    assert best["refill"] == 8
    A.save_cache({"k": {"best": best, "results": [[c, m] for c, m in res]}}, p)
    assert A.load_cache(p)["k"]["best"] == best
