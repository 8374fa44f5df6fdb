"""GPU parity of the options beyond the plain iteration, against the FP64 oracle: the
threshold variant of SIS (§2.2, last paragraph) and the "low enough error" stop (§2.3).

Bars: accepted ids and descriptors bit-exact; coefficients and RMSE within 1e-6 relative."""
import numpy as np
import pytest

from paper_2410_01752_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _thresholds(orc, sp, X, y, picks):
    """Midpoints between consecutive distinct oracle scores at the given ranks."""
    sc, va = sp.scores_all(X, y)
    u = np.unique(np.round(sc[va], 9))[::-1]
    return [0.5 * (u[r] + u[r + 1]) for r in picks if r + 1 < u.size]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["rung2", "rung3"])
def test_threshold_sis_step(S, orc, prec, case):
    """One SIS step with the threshold variant, thresholds between scores at several ranks
    (the walk ends inside the first window, after it grew, and at the cap k)."""
    if case == "rung2":
        P = inputs.workload1(0)
    else:
        P = inputs.workload2(0, N=300, d=5, sis_size=40, max_dim=2)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    for thr in _thresholds(orc, sp, P.X, P.y, [3, 17, 60]):
        k = 40
        ref = sp.sis(P.X, P.y, [], k, threshold=thr)
        with S.Sisso(P.X, P.y, P.op_set, P.rung, k, 2, precision=prec, grammar=P.grammar, sis_threshold=thr) as c:
            got = c.sis_step(P.y, [], k)
        assert got == ref, (thr, len(got), len(ref))


@pytest.mark.parametrize("prec", [0, 1])
def test_threshold_fit(S, orc, prec):
    """The whole iteration with threshold SIS (the subspace grows by fewer than k ids at some
    steps) against the oracle's iteration."""
    P = inputs.workload1(1)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    thr = _thresholds(orc, sp, P.X, P.y, [12])[0]
    ref = orc.fit(P.X, P.y, sp, P.sis_size, P.max_dim, sis_threshold=thr)
    with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=prec, sis_threshold=thr) as c:
        got = c.fit()
        assert len(got) == len(ref.dims) > 0
        for t, (g, r) in enumerate(zip(got, ref.dims)):
            assert c.sis(t + 1) == ref.sis[t]
            assert g.ids == r.ids
            np.testing.assert_allclose(g.coef, r.coef, rtol=1e-6, atol=1e-9 * np.abs(P.y).max())
            assert abs(g.rmse - r.rmse) <= 1e-6 * r.rmse


def test_threshold_above_every_score(S, orc):
    """Nothing above the threshold: no descriptor, as in the oracle."""
    P = inputs.workload1(2)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    assert orc.fit(P.X, P.y, sp, 10, 2, sis_threshold=0.9999999).dims == []
    with S.Sisso(P.X, P.y, P.op_set, P.rung, 10, 2, sis_threshold=0.9999999) as c:
        assert c.fit() == []


@pytest.mark.parametrize("prec", [0, 1])
def test_stop_rmse(S, orc, prec):
    """The iteration stops after the first step whose RMSE reaches the tolerance."""
    P = inputs.workload2(1, N=400, d=5, rung=2, sis_size=20, max_dim=4)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    full = orc.fit(P.X, P.y, sp, P.sis_size, P.max_dim)
    assert len(full.dims) == 4
    tol = 0.5 * (full.dims[1].rmse + full.dims[2].rmse)
    ref = orc.fit(P.X, P.y, sp, P.sis_size, P.max_dim, stop_rmse=tol)
    assert len(ref.dims) == 3
    with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=prec, grammar=P.grammar,
                 stop_rmse=tol) as c:
        got = c.fit()
    assert [g.ids for g in got] == [r.ids for r in ref.dims]
    for g, r in zip(got, ref.dims):
        assert abs(g.rmse - r.rmse) <= 1e-6 * r.rmse


# ---- dimensional analysis (§2.1, closing paragraph; §3.3 dimensionality) ---------------
def _units_problem(seed, N, d):
    r = np.random.default_rng(seed)
    X = r.uniform(1, 5, size=(N, d))
    y = 2.0 * (X[:, 0] - X[:, 1]) / X[:, 2] + 0.5 * X[:, 3] * X[:, 2] + 0.01 * r.normal(size=N)
    return X, y


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("labels,rung,g", [((0, 0, 1, 2), 2, 0), ((0, 0, 1, -1, 1), 2, 0), ((0, 0, 1, 2), 3, 1)])
def test_units_scores(S, orc, prec, labels, rung, g):
    """With unit labels, the screening rejects every feature that breaks the units rule
    (itself or through an operand), rejects only what the oracle rejects (the value cap is
    checked exactly by the FP64 re-score of the window, as without units), and scores the
    rest as the oracle does."""
    d = len(labels)
    X, y = _units_problem(31 + d, 120, d)
    sp = orc.Space(d, inputs.OPS9, rung, g, units=labels)
    ref, va = sp.scores_all(X, y)
    _, va_plain = orc.Space(d, inputs.OPS9, rung, g).scores_all(X, y)
    by_units = va_plain & ~va
    with S.Sisso(X, y, inputs.OPS9, rung, 10, 2, precision=prec, grammar=g, units=labels) as c:
        got = c.score_all(y, prec)
    assert by_units.sum() > 0
    assert np.all(got[by_units] < 0)
    assert np.all(va[got < 0] == False)                                  # noqa: E712
    tol = 2e-4 if prec == 1 else 1e-7
    ok = va & (got >= 0)
    assert np.abs(got[ok] - ref[ok]).max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("rung,g", [(2, 0), (3, 1)])
def test_units_fit(S, orc, prec, rung, g):
    """The whole iteration with units against the oracle's: SIS selections and descriptors
    bit-exact, coefficients within 1e-6."""
    labels = (0, 0, 1, 2)
    X, y = _units_problem(40 + rung, 200, 4)
    sp = orc.Space(4, inputs.OPS9, rung, g, units=labels)
    ref = orc.fit(X, y, sp, 15, 3)
    with S.Sisso(X, y, inputs.OPS9, rung, 15, 3, precision=prec, grammar=g, units=labels) as c:
        got = c.fit()
        assert len(got) == len(ref.dims) > 0
        for t, (a, r) in enumerate(zip(got, ref.dims)):
            assert c.sis(t + 1) == ref.sis[t]
            assert a.ids == r.ids
            np.testing.assert_allclose(a.coef, r.coef, rtol=1e-6, atol=1e-9 * np.abs(y).max())
    assert all(sp.units_of(i)[0] for s in ref.sis for i in s)


# ---- pre-screening of the primaries (§3.1; §3.3 initial_screening) ----------------------
def _wide_problem(seed, N, d):
    """A few informative primaries among many noise ones (molecular-descriptor-like width)."""
    r = np.random.default_rng(seed)
    X = r.uniform(0.5, 3.0, size=(N, d))
    X[:, 3 % d] = np.round(X[:, 3 % d], 1)                                # ties for the ranks
    y = np.log(X[:, 0]) * X[:, 1 % d] + 0.5 * X[:, 2 % d] ** 2 + 0.05 * r.normal(size=N)
    return X, y


@pytest.mark.parametrize("N,d", [(200, 30), (115, 300), (2000, 12), (333, 1)])
def test_prescreen_scores(S, orc, N, d):
    """MI within 5e-5 (FP32 kernel values, FP64 sums) and |Spearman| within 1e-12 of the
    oracle; the kept primaries equal the oracle's wherever no score is within the tolerance
    of the quantile cut."""
    X, y = _wide_problem(60 + d, N, d)
    mi_ref = orc.mi_kde(X, y)
    sp_ref = np.abs(orc.spearman(X, y))
    for method, ref, tol in ((S.PRESCREEN_MI, mi_ref, 5e-5), (S.PRESCREEN_SPEARMAN, sp_ref, 1e-12)):
        q = 0.1 if d > 10 else 1.0
        got, keep = S.prescreen(X, y, method, q)
        assert np.abs(got - ref).max() <= tol
        cut = np.quantile(ref, 1 - q) if q < 1 else -np.inf
        if np.all(np.abs(ref - cut) > 2 * tol):
            assert np.array_equal(keep, orc.prescreen_keep(ref, q))


@pytest.mark.parametrize("method", ["mi", "spearman"])
def test_prescreen_fit(S, orc, method):
    """A context built with pre-screening keeps the oracle's primaries (in their order) and
    its fit equals the oracle's fit on those columns."""
    X, y = _wide_problem(70, 300, 16)
    ref_scores = orc.mi_kde(X, y) if method == "mi" else np.abs(orc.spearman(X, y))
    keep = orc.prescreen_keep(ref_scores, 0.25)
    kept = list(np.flatnonzero(keep))
    Xk = X[:, kept]
    sp = orc.Space(len(kept), inputs.OPS9, 2)
    ref = orc.fit(Xk, y, sp, 12, 2)
    m = S.PRESCREEN_MI if method == "mi" else S.PRESCREEN_SPEARMAN
    with S.Sisso(X, y, inputs.OPS9, 2, 12, 2, prescreen=(m, 0.25)) as c:
        assert c.primaries() == kept
        got = c.fit()
        assert [g.ids for g in got] == [r.ids for r in ref.dims]
        for g, r in zip(got, ref.dims):
            np.testing.assert_allclose(g.coef, r.coef, rtol=1e-6, atol=1e-9 * np.abs(y).max())
