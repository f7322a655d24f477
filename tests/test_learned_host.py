"""Host side of the learned seed (no GPU): the cloud splits, the
oversampling rule, the committed trained weights as loaded, and the
segmentation of a re-seeded run (with a fake iteration and seeder)."""
import numpy as np
import pytest

from paper_1812_06632_gb300 import learned as L


def test_splits_are_disjoint():
    tr, va, te = set(L.TRAIN), set(L.VAL), set(L.TEST)
    assert len(tr) == len(L.TRAIN) and len(va) == len(L.VAL) and len(te) == len(L.TEST)
    assert not (tr & va) and not (tr & te) and not (va & te)


def test_seed_ranges():
    assert L.seed_ranges([]) == []
    assert L.seed_ranges([5]) == [[5, 5]]
    assert L.seed_ranges([3, 1, 2, 7, 8, 10]) == [[1, 3], [7, 8], [10, 10]]
    assert L.seed_ranges(L.TRAIN) == [[1000, 1159], [1200, 1359]]


def test_repeats_oversample_slow_clouds_up_to_the_cap():
    r = L.repeats([10, 20, 20, 40, 400])
    assert r.tolist() == [1, 1, 1, 2, 8]          # median 20: ratio rounded, at least 1, at most 8


def test_members_of_one_network_and_of_an_ensemble():
    p = L.init_params(0)
    assert L.members(p).shape == (1, p.size)
    e = np.stack([L.init_params(0), L.init_params(1)])
    m = L.members(e)
    assert m.shape == (2, p.size) and np.array_equal(m[0], p) and not np.array_equal(m[0], m[1])


def test_committed_weights_are_well_formed():
    params, norm, meta, digest = L.load_weights()
    P = L.members(params)                                   # [K, parameters], K networks averaged
    assert params.dtype == np.float32 and P.shape == (L.ENSEMBLE, L.init_params(0).size)
    assert np.all(np.isfinite(params))
    assert norm["seed_after"] in (3, 5, 10) and norm["seed_after"] == meta["seed_after"]
    assert norm["shrink"] in L.SHRINKS                      # a factor the validation sweep tried
    lo, hi, y_lo, y_hi = norm["env"]
    assert lo < hi and len(y_lo) == len(y_hi) == L.ENV_BINS
    assert all(0.0 <= a <= b for a, b in zip(y_lo, y_hi))   # the seed never lowers T (y >= 0)
    assert L.n_features(norm) == L.FEATURES               # the inputs the seeding code feeds
    for k in ("lt_std", "lr_std", "ld_std", "y_std") + (("pd_std",) if L.FEATURES == 4 else ()):
        assert norm[k] > 0.0
    assert meta["train"] == L.seed_ranges(L.TRAIN) and meta["val"] == [L.VAL[0], L.VAL[-1]]
    assert 0 <= meta["best_epoch"] < meta["epochs_run"]
    assert len(digest) == 64


class _FakeSeeder:
    """Seeds with a tenth of the latest iterate's error; records its inputs."""

    def __init__(self, history):
        self.history, self.calls = history, []

    def seeds(self, ctx, ids, Tks, Tps, Tpps=None, shrink=None):
        self.calls.append((len(ids), Tpps is not None))
        assert len(Tks) == len(Tps) == len(ids)
        assert (Tpps is not None) == (self.history == 3)
        return [t * 0.1 for t in Tks]


def _fake_iterations(monkeypatch):
    """Each dust iteration halves a cloud's error T; it has converged once
    the change, half the error, is below tol."""
    torch = pytest.importorskip("torch")

    def dust(ctx, ids, outs, seeds=None, max_iter=300, tol=0.1):
        rows = []
        for i in range(len(ids)):
            t, its, conv = float(seeds[i].item()), 0, False
            while its < max_iter and not conv:
                change = t / 2
                t -= change
                its += 1
                conv = change < tol
            outs[i].fill_(t)
            rows.append(dict(iterations=its, converged=conv, steps=its, final_max_dT=change))
        return rows
    monkeypatch.setattr(L, "dust_iterations", dust)
    return torch


@pytest.mark.parametrize("history", [2, 3])
def test_seeded_run_counts_every_segment_and_feeds_the_iterates(monkeypatch, history):
    torch = _fake_iterations(monkeypatch)
    starts = [torch.tensor([v]) for v in (1000.0, 0.15, 40.0)]
    # no re-seeding: one call, the plain count from each start
    s = _FakeSeeder(history)
    rows, fin = L.seeded_run(None, [0, 1, 2], s, starts, max_iter=300, tol=0.1)
    assert [r["iterations"] for r in rows] == [14, 1, 9] and all(r["converged"] for r in rows)
    assert s.calls == []
    # re-seeding every 5: after 5 - (history - 1) iterations and history - 1
    # single ones the unconverged clouds are seeded (error / 10) and go on
    s = _FakeSeeder(history)
    rows, fin = L.seeded_run(None, [0, 1, 2], s, starts, max_iter=300, tol=0.1, reseed=5)
    assert all(r["converged"] for r in rows)
    assert s.calls[0] == (2, history == 3)                     # clouds 0 and 2, with T_{k-2} for 3 iterates
    assert rows[1]["iterations"] == 1 and rows[0]["iterations"] < 14
    assert all(float(f.item()) < 0.2 for f in fin)
    with pytest.raises(ValueError):
        L.seeded_run(None, [0], _FakeSeeder(history), starts[:1], reseed=history - 1)
