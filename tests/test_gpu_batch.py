"""Batched multi-task form against the FP64 oracle (GPU).

Each task of the batch is an independent SISSO problem (§2.1-2.3); the persistent kernel
must reach, task by task, the oracle's descriptors (ids exact, coefficients and RMSE within
the FP32 path's tolerance), whatever the launch shape, and the same results as the
per-problem path.
"""
import json
import os

import numpy as np
import pytest

from paper_2410_01752_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workload5_oracle.jsonl")


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2410_01752_gb300 import sisso
    sisso.load()
    return sisso


def _cost(P):
    import oracle
    return oracle.Space(P.d, P.op_set, P.rung, P.grammar).sizes()[-1] * P.X.shape[0]


def _check(got, ref_dims, y, what=""):
    status, dims = got
    assert status == 0, what
    assert len(dims) == len(ref_dims), what
    for g, r in zip(dims, ref_dims):
        r_ids = r["ids"] if isinstance(r, dict) else r.ids
        r_coef = r["coef"] if isinstance(r, dict) else r.coef
        r_rmse = r["rmse"] if isinstance(r, dict) else r.rmse
        assert g.ids == list(r_ids), what
        np.testing.assert_allclose(g.coef, r_coef, rtol=1e-6, atol=1e-9 * np.abs(y).max(), err_msg=what)
        assert abs(g.rmse - r_rmse) <= 1e-6 * r_rmse + 1e-9 * y.std(), what


# tasks spanning the cost range: the cheapest, quantiles, and the most expensive
SAMPLE = [4, 311, 405, 17, 100, 230, 333, 460, 271, 115]


def test_batch_sample_vs_oracle(S, orc):
    probs = [inputs.workload5_task(p) for p in SAMPLE]
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b:
        b.run()
        res = b.results()
        st = b.stats()
    for P, p, r in zip(probs, SAMPLE, res):
        ref = orc.fit(P.X, P.y, orc.Space(P.d, P.op_set, P.rung, P.grammar), P.sis_size, P.max_dim)
        _check(r, ref.dims, P.y, f"task {p}")
    assert st["tasks_failed"] == 0
    assert st["windows_saturated"] == 0


def test_batch_full_workload_vs_oracle_golden(S):
    """All 512 tasks of the batched workload in one launch, against stored oracle results."""
    if not os.path.exists(GOLDEN):
        pytest.skip("golden file not generated")
    with open(GOLDEN) as f:
        gold = [json.loads(line) for line in f]
    probs = [inputs.workload5_task(g["task"]) for g in gold]
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b:
        b.run()
        res = b.results()
        start, end = b.timing()
        st = b.stats()
    for P, g, r in zip(probs, gold, res):
        _check(r, g["dims"], P.y, f"task {g['task']}")
    assert st["tasks_failed"] == 0 and st["windows_saturated"] == 0
    assert np.all(end >= start) and np.all(end > 0)


def test_batch_equals_single_problem_path(S):
    """The batch and the per-problem FP32 path agree task by task."""
    ps = [4, 311, 17, 230, 333]
    probs = [inputs.workload5_task(p) for p in ps]
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b:
        b.run()
        res = b.results()
    for P, r in zip(probs, res):
        with S.Sisso(P.X, P.y, P.op_set, 2, 50, 3, precision=S.PREC_FP32) as c:
            single = c.fit()
        status, dims = r
        assert status == 0 and len(dims) == len(single)
        for g, s in zip(dims, single):
            assert g.ids == s.ids
            np.testing.assert_allclose(g.coef, s.coef, rtol=1e-9, atol=1e-12 * np.abs(P.y).max())


@pytest.mark.parametrize("tune", [
    dict(score_units=1, enum_items=8, gram_rows=1, ctas_per_sm=1, window=128),
    dict(score_units=8, enum_items=512, gram_rows=8, ctas_per_sm=2, window=1024),
])
def test_batch_launch_shape_does_not_change_results(S, tune):
    ps = list(range(24))
    probs = [inputs.workload5_task(p) for p in ps]
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b:
        b.run()
        ref = b.results()
        b.tune(**tune)
        assert b.get_tune() == tune
        b.run(copies=False)
        got = b.results()
        b.run()                               # graph replay with copies
        again = b.results()
    for r, g, a in zip(ref, got, again):
        assert r[0] == g[0] == a[0] == 0
        for x, y_, z in zip(r[1], g[1], a[1]):
            assert x.ids == y_.ids == z.ids
            assert x.coef == z.coef           # same launch shape: identical
            np.testing.assert_allclose(x.coef, y_.coef, rtol=1e-12, atol=1e-12)


def test_batch_load_new_inputs(S, orc):
    """Same shapes, new values: the next copying run solves the new problems."""
    a = [inputs.workload5_task(p) for p in (4, 17)]
    with S.Batch([(P.X, P.y) for P in a], a[0].op_set, 2, 50, 3) as b:
        b.run()
        rng = np.random.default_rng(7)
        new = []
        for P in a:
            X = rng.uniform(0.5, 5.0, size=P.X.shape)
            y = 2.0 * X[:, 0] * X[:, 1] - X[:, 2] + rng.normal(0, 1e-3, size=P.X.shape[0])
            new.append((X, y))
        b.load(new)
        b.run()
        res = b.results()
    for (X, y), r in zip(new, res):
        ref = orc.fit(X, y, orc.Space(X.shape[1], a[0].op_set, 2), 50, 3)
        _check(r, ref.dims, y)


def test_batch_edge_tasks(S, orc):
    """Tiny and degenerate tasks: few samples, one primary, an exact fit that stops early."""
    rng = np.random.default_rng(3)
    X1 = rng.uniform(1, 4, size=(8, 1))
    y1 = rng.normal(size=8)
    X2 = rng.uniform(1, 4, size=(30, 3))
    y2 = 3.0 * X2[:, 0] * X2[:, 1] + 1.0                  # exact at D = 1: stops after one step
    X3 = rng.uniform(0.5, 5, size=(25, 4))
    y3 = X3[:, 0] / X3[:, 1] - 2 * X3[:, 2] ** 2 + rng.normal(0, 1e-3, size=25)
    probs = [(X1, y1), (X2, y2), (X3, y3)]
    ops = inputs.workload5_task(0).op_set
    with S.Batch(probs, ops, 2, 50, 3) as b:
        b.run()
        res = b.results()
    for (X, y), r in zip(probs, res):
        ref = orc.fit(X, y, orc.Space(X.shape[1], ops, 2), 50, 3)
        _check(r, ref.dims, y)
    assert len(res[1][1]) == 1


def test_batch_rung1_and_rung3(S, orc):
    rng = np.random.default_rng(11)
    probs = []
    for N, d in ((40, 3), (60, 4)):
        X = rng.uniform(0.5, 3, size=(N, d))
        y = X[:, 0] * X[:, 1] + np.exp(X[:, 2] / 3) + rng.normal(0, 1e-3, size=N)
        probs.append((X, y))
    ops = inputs.workload5_task(0).op_set
    for rung, k, D, ps in ((1, 5, 2, probs), (3, 10, 2, probs[:1])):
        with S.Batch(ps, ops, rung, k, D) as b:
            b.run()
            res = b.results()
        for (X, y), r in zip(ps, res):
            ref = orc.fit(X, y, orc.Space(X.shape[1], ops, rung), k, D)
            _check(r, ref.dims, y, f"rung {rung}")


def test_batch_autotune_and_cache(S, tmp_path):
    ps = list(range(16))
    probs = [inputs.workload5_task(p) for p in ps]
    cache = str(tmp_path / "tune.txt")
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b:
        b.run()
        ref = b.results()
        t1 = b.autotune(reps=1, cache_path=cache)
        b.run()
        got = b.results()
    with open(cache) as f:
        assert len(f.readlines()) == 1
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b2:
        t2 = b2.autotune(reps=1, cache_path=cache)     # cache hit: same choice, no timing
    assert t1 == t2
    for r, g in zip(ref, got):
        assert [d.ids for d in r[1]] == [d.ids for d in g[1]]


def test_fit_batch_one_shot(S, orc):
    P = inputs.workload5_task(4)
    res = S.fit_batch([(P.X, P.y)], P.op_set, 2, 50, 3)
    ref = orc.fit(P.X, P.y, orc.Space(P.d, P.op_set, 2), 50, 3)
    _check(res[0], ref.dims, P.y)


def test_wait_limit_runs_out_and_recovers(S):
    """The persistent kernel's work-queue wait is bounded: with a 1 ns no-progress limit the
    CTAs that find no work give up, the run returns SISSO_ERR_TIMEOUT once every CTA has
    returned, and with the default limit restored the next run is clean and reaches the
    oracle's stored descriptors."""
    gold = [json.loads(l) for l in open(GOLDEN)]
    ids = list(range(24))
    probs = [inputs.workload5_task(p) for p in ids]
    with S.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3) as b:
        b.set_wait_limit(1)
        with pytest.raises(S.SissoError) as e:
            b.run()
        assert e.value.status == -5
        b.set_wait_limit(0)
        b.run()
        res = b.results()
    for P, p, r in zip(probs, ids, res):
        _check(r, gold[p]["dims"], P.y, f"task {p}")
