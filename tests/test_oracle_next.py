"""Pins for the oracle's options beyond the plain iteration: the threshold variant of SIS
(§2.2, last paragraph) and the "low enough error" stop of the iteration (§2.3)."""
import numpy as np
import pytest

import brute

NAMES = ["+", "-", "*", "/", "sqrt", "^2"]


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def _tiny(seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(1, 5, size=(25, 3))
    y = X[:, 0] * X[:, 1] / X[:, 2] + 0.1 * rng.normal(size=25)
    feats, _ = brute.space(3, NAMES, 2)
    values = [brute.evaluate(f, X) for f in feats]
    ok = [brute.valid(v, f, X) for v, f in zip(values, feats)]
    return X, y, values, ok


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_threshold_sis_matches_brute_force(orc, seed):
    """Thresholds between scores, on y and on a residual with a prior S: the oracle's walk
    equals the brute-force walk that ends at the first maximum at or below the threshold."""
    X, y, values, ok = _tiny(seed)
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    sc = np.sort(np.unique(np.round([brute.abs_corr(v, y) for v, o in zip(values, ok) if o], 12)))[::-1]
    for thr in (0.5 * (sc[3] + sc[4]), 0.5 * (sc[12] + sc[13]), 0.5 * (sc[30] + sc[31])):
        acc = sp.sis(X, y, [], 40, threshold=thr)
        ref = brute.sis(values, y, [], 40, ok, thr)
        assert acc == ref
        assert 0 < len(acc) < 40
        # every accepted feature scores above the threshold
        assert all(brute.abs_corr(values[i], y) > thr for i in acc)
    acc1 = sp.sis(X, y, [], 5)
    v = values[acc1[0]]
    r = y - np.polyval(np.polyfit(v, y, 1), v)
    thr = 0.2
    assert sp.sis(X, r, acc1, 40, threshold=thr) == brute.sis(values, r, acc1, 40, ok, thr)


def test_threshold_zero_and_above_all(orc):
    """Threshold 0 is the plain top-k step; a threshold above every score accepts nothing
    and a fit with it ends with no descriptor."""
    X, y, values, ok = _tiny(4)
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    assert sp.sis(X, y, [], 12, threshold=0.0) == sp.sis(X, y, [], 12)
    assert sp.sis(X, y, [], 12, threshold=1.0) == []
    res = orc.fit(X, y, sp, 5, 2, sis_threshold=1.0)
    assert res.dims == [] and res.sis in ([], [[]])


@pytest.mark.parametrize("seed", [5, 6])
def test_threshold_fit_matches_brute_force(orc, seed):
    """The whole iteration with threshold SIS equals the brute-force iteration."""
    X, y, values, ok = _tiny(seed)
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    thr = 0.3
    ref = brute.sisso(X, y, 3, NAMES, 2, 30, 3, thr=thr)
    res = orc.fit(X, y, sp, 30, 3, sis_threshold=thr)
    assert len(res.dims) == len(ref) > 0
    for t, (tup, c, rmse, S) in enumerate(ref):
        assert res.dims[t].ids == tup
        assert np.allclose(res.dims[t].coef, c, rtol=1e-8, atol=1e-10)
        assert sum(res.sis[: t + 1], []) == S


def test_stop_rmse_ends_the_iteration(orc):
    """With the tolerance set between the RMSE of the 2-term and the 1-term model, the
    iteration stops after 2 terms with the full iteration's first two models; the
    brute-force iteration stops at the same place."""
    X, y, values, ok = _tiny(7)
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    full = orc.fit(X, y, sp, 8, 3)
    assert len(full.dims) == 3 and full.dims[1].rmse < full.dims[0].rmse
    tol = 0.5 * (full.dims[0].rmse + full.dims[1].rmse)
    short = orc.fit(X, y, sp, 8, 3, stop_rmse=tol)
    assert len(short.dims) == 2
    for a, b in zip(short.dims, full.dims[:2]):
        assert a.ids == b.ids and a.coef == b.coef and a.rmse == b.rmse
    ref = brute.sisso(X, y, 3, NAMES, 2, 8, 3, stop_rmse=tol)
    assert [r[0] for r in ref] == [d.ids for d in short.dims]


# ---- dimensional analysis (§2.1, closing paragraph; §3.3 dimensionality) ---------------
ALL12 = brute.TABLE


OPS_R3 = ["+", "-", "*", "/", "exp", "sqrt", "^-1"]


@pytest.mark.parametrize("labels,rung,nxp,ops", [((0, 0, 1), 2, False, ALL12), ((0, 1, -1), 2, False, ALL12),
                                                 ((1, 1), 3, False, OPS_R3), ((0, 1), 3, True, OPS_R3)])
def test_units_match_brute_force(orc, labels, rung, nxp, ops):
    """Every feature's unit exponents and consistency flag equal the brute-force units of
    its expression tree (exact fractions)."""
    d = len(labels)
    feats, sizes = brute.space(d, ops, rung, nxp)
    sp = orc.Space(d, _mask(orc, ops), rung, orc.GRAMMAR_NEW_X_PREV if nxp else orc.GRAMMAR_EQ2, units=labels)
    assert sp.sizes() == sizes
    n_bad = 0
    for i, f in enumerate(feats):
        u = brute.units(f, labels)
        ok, e = sp.units_of(i)
        assert ok == (u is not None), brute.to_str(f)
        if ok:
            assert {k: v for k, v in enumerate(e) if v} == {k: int(v * 16) for k, v in u.items()}, brute.to_str(f)
        n_bad += not ok
    assert n_bad > 0


def test_units_validity_and_sis_match_brute_force(orc):
    """With units, a feature is valid iff its values are valid and it (with every operand) is
    dimensionally consistent; the SIS step with units equals the brute-force walk over
    those features."""
    rng = np.random.default_rng(21)
    X = rng.uniform(1, 5, size=(30, 3))
    y = (X[:, 0] - X[:, 1]) / X[:, 2] + 0.05 * rng.normal(size=30)
    labels = (0, 0, 1)
    feats, _ = brute.space(3, ALL12, 2)
    values = [brute.evaluate(f, X) for f in feats]
    ok = [brute.valid(v, f, X) and brute.units(f, labels) is not None for v, f in zip(values, feats)]
    sp = orc.Space(3, _mask(orc, ALL12), 2, units=labels)
    sc, va = sp.scores_all(X, y)
    assert list(va) == ok
    for i in np.flatnonzero(va):
        assert sc[i] == pytest.approx(brute.abs_corr(values[i], y), abs=1e-12)
    assert sp.sis(X, y, [], 15) == brute.sis(values, y, [], 15, ok)


def test_units_fit_recovers_physical_descriptor(orc):
    """y = 2 (x1 - x2) / x3 + 1 with x1, x2 lengths and x3 a time: the units-aware fit finds
    (x1-x2)/x3 as its 1-term descriptor, its whole iteration equals the brute-force one
    over the consistent features, and no selected feature breaks the units rule."""
    rng = np.random.default_rng(22)
    X = rng.uniform(1, 5, size=(40, 3))
    y = 2.0 * (X[:, 0] - X[:, 1]) / X[:, 2] + 1.0
    labels = (0, 0, 1)
    sp = orc.Space(3, _mask(orc, ALL12), 2, units=labels)
    res = orc.fit(X, y, sp, 10, 2)
    v = sp.eval(X, res.dims[0].ids[0])                  # (x1-x2)/x3 or a duplicate of it
    assert abs(np.corrcoef(v, (X[:, 0] - X[:, 1]) / X[:, 2])[0, 1]) > 1 - 1e-12
    assert res.dims[0].rmse < 1e-9
    assert all(sp.units_of(i)[0] for s in res.sis for i in s)


def test_dimensionless_units_change_nothing(orc):
    """All primaries dimensionless: every rule is met, so validity and scores equal those of
    the space without units."""
    rng = np.random.default_rng(23)
    X = rng.uniform(0.5, 3, size=(25, 3))
    y = rng.normal(size=25)
    a = orc.Space(3, _mask(orc, ALL12), 2).scores_all(X, y)
    b = orc.Space(3, _mask(orc, ALL12), 2, units=(-1, -1, -1)).scores_all(X, y)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])


# ---- pre-screening of the primaries (§3.1; §3.3 initial_screening) ----------------------
def _mi_scipy(a, b):
    st = pytest.importorskip("scipy.stats")
    kxy, kx, ky = st.gaussian_kde(np.vstack([a, b])), st.gaussian_kde(a), st.gaussian_kde(b)
    return float(np.mean(np.log(kxy(np.vstack([a, b])) / (kx(a) * ky(b)))))


def test_mi_kde_equals_library_kde(orc):
    """The oracle's MI is the resubstitution estimate built from scipy's Gaussian KDE
    (Scott's rule, full joint covariance), for linear, monotone, periodic and independent
    relations and heavy-tailed inputs."""
    r = np.random.default_rng(50)
    N = 400
    x = r.normal(size=N)
    y = np.sin(2 * x) + 0.3 * r.normal(size=N)
    X = np.column_stack([x, np.exp(x), r.standard_t(3, size=N), x ** 2, r.uniform(size=N)])
    mi = orc.mi_kde(X, y)
    for i in range(X.shape[1]):
        assert mi[i] == pytest.approx(_mi_scipy(X[:, i], y), rel=1e-10, abs=1e-12)


def test_mi_kde_gaussian_closed_form_and_invariances(orc):
    """Bivariate normal pairs: within 0.03 of MI = -log(1 - rho^2)/2 at N = 3000 and ordered
    by rho; the estimate is symmetric in (x, y) and unchanged by an affine map of x."""
    N = 3000
    r = np.random.default_rng(51)
    g = r.normal(size=(N, 3))
    y = r.normal(size=N)
    rhos = (0.5, 0.8, 0.95)
    X = np.column_stack([rho * y + np.sqrt(1 - rho ** 2) * g[:, i] for i, rho in enumerate(rhos)])
    mi = orc.mi_kde(X, y)
    for m, rho in zip(mi, rhos):
        assert abs(m - (-0.5 * np.log(1 - rho ** 2))) <= 0.03
    assert mi[0] < mi[1] < mi[2]
    assert orc.mi_kde(y[:, None], X[:, 1])[0] == pytest.approx(mi[1], rel=1e-12)
    assert orc.mi_kde(3.0 * X[:, 1:2] - 7.0, y)[0] == pytest.approx(mi[1], rel=1e-9)


def test_spearman_equals_library(orc):
    """Spearman rank correlation with average ranks for ties equals scipy's."""
    st = pytest.importorskip("scipy.stats")
    r = np.random.default_rng(52)
    N = 200
    y = r.normal(size=N)
    X = np.column_stack([np.exp(y) + 0.1 * r.normal(size=N), r.integers(0, 5, size=N).astype(float),
                         -y ** 3, r.normal(size=N)])
    rho = orc.spearman(X, np.round(y, 1))
    for i in range(X.shape[1]):
        assert rho[i] == pytest.approx(st.spearmanr(X[:, i], np.round(y, 1)).statistic, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("d,q", [(10, 0.3), (1445, 0.01), (7, 1.0), (50, 0.5)])
def test_prescreen_keep_is_top_quantile(orc, d, q):
    """Kept primaries are those scoring strictly above numpy's (1 - q)-quantile."""
    s = np.random.default_rng(d).uniform(size=d)
    keep = orc.prescreen_keep(s, q)
    if q >= 1.0:
        assert keep.all()
    else:
        assert np.array_equal(keep, s > np.quantile(s, 1.0 - q))
        assert 0 < keep.sum() <= int(np.ceil(q * d))
