"""Resampled fits through the batched form (§2.4 closing paragraphs; §4.5 ensemble): every
task against the FP64 oracle's fit of the same rows, and the combined quantities (bagged
prediction, pooled held-out RMSE) against the same combination of the oracle's models.

Bars: descriptors bit-exact; coefficients within 1e-6 relative; combined quantities within
1e-6 relative."""
import numpy as np
import pytest

from paper_2410_01752_gb300 import ensemble, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _oracle_models(orc, sp, X, y, row_sets, k, D):
    return [orc.fit(X[r], y[r], sp, k, D) for r in row_sets]


def _oracle_pred(sp, X, dim):
    return dim.coef[0] + sum(c * sp.eval(X, i) for c, i in zip(dim.coef[1:], dim.ids))


def _same(models, ref, y):
    for m, r in zip(models, ref):
        assert m.status == 0
        assert [d.ids for d in m.dims] == [d.ids for d in r.dims]
        for a, b in zip(m.dims, r.dims):
            np.testing.assert_allclose(a.coef, b.coef, rtol=1e-6, atol=1e-9 * np.abs(y).max())


def test_kfold_matches_oracle(S, orc):
    P = inputs.workload1(3, N=160)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    cv = ensemble.kfold(P.X, P.y, P.op_set, P.rung, 10, 3, K=4, seed=2)
    ref = _oracle_models(orc, sp, P.X, P.y, [tr for tr, _ in cv.folds], 10, 3)
    _same(cv.models, ref, P.y)
    for t in range(1, 4):
        sq = []
        for (_, te), r in zip(cv.folds, ref):
            e = P.y[te] - _oracle_pred(sp, P.X, r.dims[t - 1])[te]
            sq.append(e * e)
        assert cv.rmse[t - 1] == pytest.approx(float(np.sqrt(np.mean(np.concatenate(sq)))), rel=1e-6)
    # the planted one-term model (3 x1 x2 / x3 + 0.5, noise sd 0.01): held-out error at the
    # noise level for t = 1, larger for the over-fitted t = 2, 3
    assert int(np.argmin(cv.rmse)) == 0 and cv.rmse[0] < 0.015


def test_bagging_matches_oracle(S, orc):
    P = inputs.workload5_task(7)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    bag = ensemble.bagging(P.X, P.y, P.op_set, P.rung, 12, 2, n_models=6, seed=4)
    rows = ensemble.bootstrap_rows(P.N, 6, seed=4)
    assert all(np.array_equal(m.rows, r) for m, r in zip(bag.models, rows))
    ref = _oracle_models(orc, sp, P.X, P.y, rows, 12, 2)
    _same(bag.models, ref, P.y)
    want = np.mean([_oracle_pred(sp, P.X, r.dims[-1]) for r in ref], axis=0)
    np.testing.assert_allclose(bag.prediction, want, rtol=1e-6, atol=1e-9 * np.abs(P.y).max())
    assert sum(bag.descriptor_counts.values()) == 6


def test_partition_ensemble_matches_oracle(S, orc):
    """The §4.5 ensemble at reduced count: 10 disjoint subsets of 100 samples of the
    four-term problem, k = 20, D <= 4, in one launch."""
    P = inputs.ensemble_problem(0, N=1000)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    rows = ensemble.partition_rows(P.N, 10, 100, seed=0)
    models = ensemble.fit_rows(P.X, P.y, rows, P.op_set, P.rung, P.sis_size, P.max_dim)
    ref = _oracle_models(orc, sp, P.X, P.y, rows, P.sis_size, P.max_dim)
    _same(models, ref, P.y)


def test_ensemble_full_against_golden(S):
    """The full §4.5 ensemble: the 30 disjoint 100-sample subsets of the 3000-sample problem
    in one launch, every model equal to the oracle's stored fit
    (tests/golden/ensemble_oracle.json, written from the oracle alone)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ensemble_oracle.json")))
    P = inputs.ensemble_problem(0)
    rows = inputs.partition_rows(P.N, 30, 100, 0)
    models = ensemble.fit_rows(P.X, P.y, rows, P.op_set, P.rung, P.sis_size, P.max_dim)
    assert len(models) == len(gold) == 30
    for m, rec in zip(models, gold):
        assert m.status == 0
        assert [d.ids for d in m.dims] == [g["ids"] for g in rec["dims"]]
        for d, g in zip(m.dims, rec["dims"]):
            np.testing.assert_allclose(d.coef, g["coef"], rtol=1e-6, atol=1e-9 * np.abs(P.y).max())
            assert abs(d.rmse - g["rmse"]) <= 1e-6 * g["rmse"]
