"""bench.py's reference arm runs the oracle on the host (no GPU): its JSON
line carries the keys of the bench contract."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--cpu-sample", "64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "photon-cell steps/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_map_segment_count_matches_brute_force():
    """The segment count bench.py divides by (leaf crossings of every pixel's
    ray through a regular grid) against marching each ray in small steps.
    A crossing through an edge or corner counts once per plane crossed, as
    the traversal does (it takes one face at a time, the second step of zero
    length)."""
    sys.path.insert(0, ROOT)
    import bench
    n = 6
    d = np.array([1.0, 0.7, 0.4]); d /= np.linalg.norm(d)
    up = np.array([0.0, 0.0, 1.0])
    e1 = np.cross(up, d); e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    c = np.array([3.0, 3.0, 3.0])
    npx = npy = 9
    pix = 1.1
    segs, rays = bench._map_segments(n, d, e1, e2, c, npx, npy, pix)
    total, hit = 0, 0
    for py in range(npy):
        for px in range(npx):
            o = c + ((px + 0.5) - npx / 2) * pix * e1 + ((py + 0.5) - npy / 2) * pix * e2
            ts = np.arange(-20.0, 20.0, 1e-3)
            pts = o[None, :] + ts[:, None] * d[None, :]
            inside = np.all((pts >= 0) & (pts < n), axis=1)
            if not inside.any():
                continue
            cells = np.floor(pts[inside]).astype(int)
            total += 1 + int((np.diff(cells, axis=0) != 0).sum())
            hit += 1
    assert rays == hit and segs == total


def test_gpus_flag_launches_one_process_per_rank():
    """`bench.py --gpus 2` outside torchrun relaunches itself under
    torch.distributed.run with two ranks; the reference arm then runs on rank
    0 alone, which reports the launch's world size."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "1", "--cpu-sample", "32"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600, env={k: v for k, v in os.environ.items() if k != "WORLD_SIZE"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1                       # rank 1 prints nothing
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
