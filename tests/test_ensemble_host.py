"""Row sets of the resampled fits (host logic, no GPU): disjoint partitions, bootstrap
samples and k folds, each seeded and reproducible."""
import numpy as np
import pytest

from paper_2410_01752_gb300 import ensemble


def test_partition_rows_disjoint():
    rows = ensemble.partition_rows(3000, 30, 100, seed=5)
    assert len(rows) == 30 and all(r.size == 100 for r in rows)
    allr = np.concatenate(rows)
    assert np.unique(allr).size == 3000 and allr.min() == 0 and allr.max() == 2999
    assert all(np.all(np.diff(r) > 0) for r in rows)
    again = ensemble.partition_rows(3000, 30, 100, seed=5)
    assert all(np.array_equal(a, b) for a, b in zip(rows, again))
    with pytest.raises(ValueError):
        ensemble.partition_rows(100, 3, 40, seed=0)


def test_bootstrap_rows():
    rows = ensemble.bootstrap_rows(500, 8, seed=3)
    assert len(rows) == 8 and all(r.size == 500 for r in rows)
    assert all(r.min() >= 0 and r.max() < 500 for r in rows)
    # with replacement: about 1 - 1/e of the rows appear in a sample
    frac = np.mean([np.unique(r).size / 500 for r in rows])
    assert 0.58 < frac < 0.68
    assert not np.array_equal(rows[0], rows[1])
    assert all(np.array_equal(a, b) for a, b in zip(rows, ensemble.bootstrap_rows(500, 8, seed=3)))
    assert ensemble.bootstrap_rows(500, 2, seed=3, size=50)[0].size == 50


@pytest.mark.parametrize("N,K", [(10, 2), (103, 5), (160, 4), (7, 7)])
def test_kfold_rows(N, K):
    folds = ensemble.kfold_rows(N, K, seed=11)
    assert len(folds) == K
    tests = [te for _, te in folds]
    assert np.array_equal(np.sort(np.concatenate(tests)), np.arange(N))       # a partition
    sizes = sorted(te.size for te in tests)
    assert sizes[-1] - sizes[0] <= 1
    for tr, te in folds:
        assert np.intersect1d(tr, te).size == 0 and tr.size + te.size == N
    with pytest.raises(ValueError):
        ensemble.kfold_rows(5, 1, seed=0)
