"""Pins for the oracle's whole SISSO iteration (§2.3 Eq. 8, §3.3 outputs)."""
import numpy as np
import pytest

import brute

ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


@pytest.mark.parametrize("seed,names,rung,k,T,nxp", [
    (0, ["+", "-", "*", "/", "sqrt"], 2, 4, 3, False),
    (1, ["+", "*", "/", "log", "^2"], 2, 3, 3, False),
    (2, ["+", "*", "exp-"], 3, 3, 2, False),
    (3, ["+", "-", "*", "/", "log"], 3, 4, 3, True),      # the restricted rung-3 grammar
])
def test_fit_matches_brute_force_pipeline(orc, seed, names, rung, k, T, nxp):
    """Every step (S_t, descriptor, coefficients, RMSE) equals the numpy brute-force
    iteration: SIS on y, then on the residual of the best lstsq fit."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(1, 5, size=(20, 2 if rung == 3 else 3))
    d = X.shape[1]
    y = 2 * X[:, 0] / X[:, 1] + np.sqrt(X[:, -1]) + 0.05 * rng.normal(size=20)
    ref = brute.sisso(X, y, d, names, rung, k, T, new_x_prev=nxp)
    res = orc.fit(X, y, orc.Space(d, _mask(orc, names), rung, orc.GRAMMAR_NEW_X_PREV if nxp else orc.GRAMMAR_EQ2),
                  k, T)
    assert len(res.dims) == len(ref)
    for t, (tup, c, rmse, S) in enumerate(ref):
        assert res.dims[t].ids == tup
        assert np.allclose(res.dims[t].coef, c, rtol=1e-8, atol=1e-10)
        assert res.dims[t].rmse == pytest.approx(rmse, rel=1e-8)
        assert sum(res.sis[: t + 1], []) == S


def test_planted_noise_free_recovery(orc):
    """y = c*x1*x2/x3 + c0 without noise: the 1-term descriptor is x1*x2/x3 (lowest id
    among its duplicates), c and c0 to 1e-10, RMSE ~ 0, and the iteration stops there."""
    rng = np.random.default_rng(42)
    X = rng.uniform(1, 5, size=(50, 5))
    y = 3.0 * X[:, 0] * X[:, 1] / X[:, 2] + 0.5
    sp = orc.Space(5, _mask(orc, ALL9), 2)
    res = orc.fit(X, y, sp, 20, 3)
    assert len(res.dims) == 1
    d1 = res.dims[0]
    f = sp.eval(X, d1.ids[0])
    assert np.allclose(f, X[:, 0] * X[:, 1] / X[:, 2], rtol=1e-13)
    assert d1.coef[1] == pytest.approx(3.0, abs=1e-10)
    assert d1.coef[0] == pytest.approx(0.5, abs=1e-10)
    assert d1.rmse <= 1e-12 * y.std()
    assert d1.r2 == pytest.approx(1.0, abs=1e-15)


def test_best_subset_special_case(orc):
    """When k*T covers every distinct valid feature, SISSO's t-term result is the best
    t-subset over all of phi (brute force over distinct valid features)."""
    rng = np.random.default_rng(3)
    X = rng.uniform(1, 5, size=(15, 2))
    y = X[:, 0] ** 2 - 3 * X[:, 1] + 0.3 * rng.normal(size=15)
    names = ["+", "*", "^2", "sqrt"]
    feats, _ = brute.space(2, names, 1)
    vals = [brute.evaluate(f, X) for f in feats]
    distinct = []
    for i, v in enumerate(vals):
        z = brute.standardise(v)
        if brute.valid(v) and not any(np.max(np.abs(z - brute.standardise(vals[j]))) <= 1e-8
                                      or np.max(np.abs(z + brute.standardise(vals[j]))) <= 1e-8
                                      for j in distinct):
            distinct.append(i)
    res = orc.fit(X, y, orc.Space(2, _mask(orc, names), 1), len(feats), 2)
    assert sorted(sum(res.sis, [])) == sorted(distinct)
    for t in (1, 2):
        cols = np.column_stack([vals[i] for i in distinct])
        (rss, tup, _), _ = brute.best_subset(cols, y, t, distinct)
        assert res.dims[t - 1].ids == list(tup)
        assert res.dims[t - 1].rmse == pytest.approx(np.sqrt(rss / 15), rel=1e-9)


def test_affine_and_permutation_invariance(orc):
    """y -> a*y + b keeps the descriptors and scales the coefficients; permuting the
    samples changes nothing."""
    rng = np.random.default_rng(8)
    X = rng.uniform(1, 5, size=(40, 4))
    y = X[:, 0] * X[:, 3] - np.log(X[:, 1]) + 0.05 * rng.normal(size=40)
    sp = orc.Space(4, _mask(orc, ALL9), 2)
    base = orc.fit(X, y, sp, 8, 2)
    a, b = -2.5, 7.0
    aff = orc.fit(X, a * y + b, sp, 8, 2)
    perm = rng.permutation(40)
    prm = orc.fit(X[perm], y[perm], sp, 8, 2)
    for t in range(2):
        assert aff.dims[t].ids == base.dims[t].ids == prm.dims[t].ids
        cb = np.array(base.dims[t].coef)
        ca = np.array(aff.dims[t].coef)
        assert np.allclose(ca[1:], a * cb[1:], rtol=1e-8)
        assert ca[0] == pytest.approx(a * cb[0] + b, rel=1e-8)
        assert np.allclose(prm.dims[t].coef, cb, rtol=1e-8)
        assert aff.dims[t].rmse == pytest.approx(abs(a) * base.dims[t].rmse, rel=1e-8)


def test_rmse_non_increasing_and_subset_counts(orc):
    """RSS is non-increasing in t, and step t examines C(|S_t|, t) subsets."""
    import math
    rng = np.random.default_rng(4)
    X = rng.uniform(1, 5, size=(60, 4))
    y = np.exp(X[:, 0] / 5) + X[:, 1] * X[:, 2] + 0.1 * rng.normal(size=60)
    res = orc.fit(X, y, orc.Space(4, _mask(orc, ALL9), 2), 10, 3)
    n = 0
    for t, dm in enumerate(res.dims, start=1):
        n += len(res.sis[t - 1])
        assert dm.subsets == math.comb(n, t)
        if t > 1:
            assert dm.rmse <= res.dims[t - 2].rmse + 1e-12


@pytest.mark.parametrize("row,expr,names,T,k", [
    # Table 1 rows reachable at rung 2 (§4.1: x in [1,5]^d, Gaussian noise sd 0.05)
    (2, lambda X: 2 * np.sin(X[:, 1]) + 3 * np.sqrt(X[:, 0]), ["+", "*", "sin", "sqrt"], 2, 20),
    (4, lambda X: 3 * X[:, 2] + X[:, 1] ** 2 + X[:, 0] ** 3, ["+", "*", "^2", "^3"], 3, 20),
    (8, lambda X: 5 * X[:, 0] * X[:, 2] ** 2 + X[:, 0] ** 3 + 3 * X[:, 0] * X[:, 1] ** 2,
     ["+", "*", "^2", "^3"], 3, 100),
])
def test_table1_recovery_qualitative(orc, row, expr, names, T, k):
    """Qualitative: the planted structures of Table 1 rows 2, 4, 8 are recovered (the
    fitted model reproduces the noise-free target to the noise level).  SISSO is a
    heuristic: row 8 needs a wider screen (k = 100) on this draw."""
    rng = np.random.default_rng(100 + row)
    d = 3 if row != 2 else 2
    X = rng.uniform(1, 5, size=(60, d))
    clean = expr(X)
    y = clean + 0.05 * rng.normal(size=60)
    sp = orc.Space(d, _mask(orc, names), 2)
    res = orc.fit(X, y, sp, k, T)
    dm = res.dims[-1]
    yhat = dm.coef[0] + sum(c * sp.eval(X, i) for c, i in zip(dm.coef[1:], dm.ids))
    assert np.sqrt(np.mean((yhat - clean) ** 2)) < 0.05
