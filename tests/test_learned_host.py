"""Host side of the learned seed (no GPU): the cloud splits, the
oversampling rule, and the committed trained weights as loaded."""
import numpy as np

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
