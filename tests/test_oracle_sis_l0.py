"""Pins for the oracle's SIS step (§2.2 Eqs. 5-6) and exhaustive l0 (§2.3 Eqs. 7-8)."""
import math

import numpy as np
import pytest

import brute

ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def test_scores_match_numpy_corrcoef(orc):
    """|rho| of every valid feature equals |numpy.corrcoef| of independently evaluated
    values; invalid flags follow the validity rule."""
    rng = np.random.default_rng(11)
    X = rng.uniform(-2, 5, size=(40, 3))          # negatives: log/sqrt domain errors
    y = rng.normal(size=40)
    feats, sizes = brute.space(3, ALL9, 2)
    sp = orc.Space(3, _mask(orc, ALL9), 2)
    sc, va = sp.scores(X, y)
    n_invalid = 0
    for i, f in enumerate(feats):
        v = brute.evaluate(f, X)
        assert va[i] == brute.valid(v, f, X), brute.to_str(f)
        if va[i]:
            assert sc[i] == pytest.approx(brute.abs_corr(v, y), abs=1e-12)
        else:
            n_invalid += 1
    assert n_invalid > 0


def test_near_constant_and_cap_are_invalid(orc):
    """(x1/x2)*(x2/x1) == 1 (near-constant) and exp(exp(x)) > 1e12 are invalid."""
    X = np.random.default_rng(2).uniform(3.0, 5.0, size=(30, 2))
    sp = orc.Space(2, _mask(orc, ["*", "/", "exp"]), 2)
    names = {sp.expr(i): i for i in range(sp.n_features)}
    sc, va = sp.scores(X, X[:, 0])
    assert not va[names["((x1/x2)*(x2/x1))"]]
    assert not va[names["exp(exp(x1))"]]          # e^{e^3} = 5e8 .. e^{e^5} = 3e64
    assert va[names["exp(x1)"]]


@pytest.mark.parametrize("seed,k", [(0, 5), (1, 12), (2, 30)])
def test_sis_matches_brute_force(orc, seed, k):
    """SIS on a tiny space equals the brute-force walk (numpy corrcoef scores, the
    tie-tolerant order, duplicates up to sign) both on y and with a prior S."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(1, 5, size=(25, 3))
    y = X[:, 0] * X[:, 1] / X[:, 2] + 0.1 * rng.normal(size=25)
    names = ["+", "-", "*", "/", "sqrt", "^2"]
    feats, _ = brute.space(3, names, 2)
    values = [brute.evaluate(f, X) for f in feats]
    ok = [brute.valid(v, f, X) for v, f in zip(values, feats)]
    sp = orc.Space(3, _mask(orc, names), 2)
    acc1 = sp.sis(X, y, [], k)
    assert acc1 == brute.sis(values, y, [], k, ok)
    r = y - np.polyval(np.polyfit(values[acc1[0]], y, 1), values[acc1[0]])
    acc2 = sp.sis(X, r, acc1, k)
    assert acc2 == brute.sis(values, r, acc1, k, ok)
    assert not set(acc1) & set(acc2)


def test_identically_zero_features_are_invalid(orc):
    """Features whose root + or - cancels exactly (x1-(x3+(x1-x3)), x1*x2-(x2*x4)/(x4/x1))
    are invalid, whatever score their rounding noise would get; a small but genuine
    difference of nearly collinear primaries stays valid."""
    rng = np.random.default_rng(6)
    X = rng.lognormal(0, 0.5, size=(60, 4))
    y = rng.normal(size=60)
    names = ["+", "-", "*", "/"]
    sp = orc.Space(4, _mask(orc, names), 3, orc.GRAMMAR_NEW_X_PREV)
    ids = {sp.expr(i): i for i in range(sp.n_features)}
    zero = ["(x1-(x3+(x1-x3)))", "((x1*x2)-((x2*x4)/(x4/x1)))"]
    sc, va = sp.scores(X, y, [ids[e] for e in zero])
    assert not va.any()
    for e in zero:                          # their values really are rounding noise
        v = sp.eval(X, ids[e])
        assert np.abs(v).max() < 1e-13
    Xc = X.copy()
    Xc[:, 1] = Xc[:, 0] + 1e-4 * rng.normal(size=60)   # corr ~ 0.99999
    sc, va = sp.scores(Xc, y, [ids["(x1-x2)"]])
    assert va.all()


def test_validity_is_recursive(orc):
    """A feature built from an invalid feature is invalid: log(x2*x2^-1) (log of a
    constant) and (exp(x1))^-1 where exp(x1) exceeds 1e12 although 1/exp(x1) does not."""
    rng = np.random.default_rng(12)
    X = rng.uniform(1, 5, size=(40, 2))
    X[7, 0] = 30.0                                   # exp(30) = 1.07e13 > 1e12
    sp = orc.Space(2, _mask(orc, ["*", "exp", "log", "^-1"]), 3)
    ids = {sp.expr(i): i for i in range(sp.n_features)}
    sc, va = sp.scores(X, rng.normal(size=40), [ids[e] for e in ("log((x2*(x2)^-1))", "(exp(x1))^-1",
                                                                  "exp(x1)", "(x2)^-1", "log((x1*x2))")])
    assert list(va) == [False, False, False, True, True]
    assert np.abs(1.0 / np.exp(X[:, 0])).max() < 1e12     # its own values are fine


def test_sis_duplicates_are_skipped(orc):
    """Value-identical features (x1*(x2/x3), (x1*x2)/x3, ...) enter S once, as the
    lowest id; sign-flipped duplicates too."""
    X = np.random.default_rng(5).uniform(1, 5, size=(50, 3))
    y = 3 * X[:, 0] * X[:, 1] / X[:, 2]
    sp = orc.Space(3, _mask(orc, ["*", "/", "-"]), 2)
    acc = sp.sis(X, y, [], 10)
    Z = np.array([brute.standardise(sp.eval(X, i)) for i in acc])
    for a in range(len(acc)):
        for b in range(a):
            assert min(np.abs(Z[a] - Z[b]).max(), np.abs(Z[a] + Z[b]).max()) > 1e-8
    dup_ids = [i for i in range(sp.n_features)
               if np.allclose(brute.standardise(sp.eval(X, i)) if brute.valid(sp.eval(X, i)) else 0,
                              Z[0], atol=1e-8)]
    assert acc[0] == min(dup_ids) and len(dup_ids) > 1


def _gram(cols, y):
    Z = (cols - cols.mean(0)) / cols.std(0)
    yc = y - y.mean()
    N = len(y)
    return Z.T @ Z / N, Z.T @ yc / N, float(yc @ yc) / N


@pytest.mark.parametrize("n,D,seed", [(8, 1, 0), (10, 2, 1), (12, 3, 2), (9, 4, 3), (16, 3, 4), (11, 5, 5),
                                      (14, 5, 6)])
def test_l0_matches_lstsq_brute_force(orc, n, D, seed):
    """Exhaustive l0 equals numpy.linalg.lstsq over every D-subset (with intercept):
    the same winner, the same RSS, C(n, D) subsets examined."""
    rng = np.random.default_rng(seed)
    N = 30
    cols = rng.normal(size=(N, n)) + 0.3 * rng.normal(size=(N, 1))
    y = cols[:, :D] @ rng.uniform(-2, 2, D) + 0.2 * rng.normal(size=N)
    gid = list(rng.permutation(1000)[:n])
    G, b, syy = _gram(cols, y)
    pos, rss, ex = orc.l0(G, b, syy, N, D, gid)
    (rss_bf, tup_bf, sub_bf), count = brute.best_subset(cols, y, D, gid)
    assert ex == count == math.comb(n, D)
    assert tuple(sorted(gid[p] for p in pos)) == tup_bf
    assert rss == pytest.approx(rss_bf, rel=1e-9, abs=1e-9)
    # the winner's RSS is <= that of every other subset
    import itertools
    for sub in itertools.combinations(range(n), D):
        assert brute.rss_with_intercept(cols[:, sub], y) >= rss - 1e-9


def test_l0_d1_closed_form(orc):
    """D = 1: RSS = SST (1 - rho^2) of the best single feature."""
    rng = np.random.default_rng(7)
    N, n = 60, 9
    cols = rng.normal(size=(N, n))
    y = 2 * cols[:, 4] + rng.normal(size=N)
    G, b, syy = _gram(cols, y)
    pos, rss, _ = orc.l0(G, b, syy, N, 1, list(range(n)))
    rho = np.array([np.corrcoef(cols[:, j], y)[0, 1] for j in range(n)])
    sst = float(((y - y.mean()) ** 2).sum())
    assert pos == [int(np.argmax(rho ** 2))]
    assert rss == pytest.approx(sst * (1 - rho[pos[0]] ** 2), rel=1e-10)


def test_l0_singular_subsets_skipped_and_ties(orc):
    """Collinear pairs (pivot <= 1e-12) are skipped; exact RSS ties go to the smallest
    ascending global-id tuple."""
    rng = np.random.default_rng(9)
    N = 40
    a, c = rng.normal(size=N), rng.normal(size=N)
    cols = np.column_stack([a, 2 * a + 1, c, -a])  # 0, 1 and 3 are collinear
    y = a + 0.5 * c
    G, b, syy = _gram(cols, y)
    pos, rss, _ = orc.l0(G, b, syy, N, 2, [40, 30, 20, 10])
    assert rss == pytest.approx(0.0, abs=1e-9)
    # {0,2}, {1,2} and {3,2} all fit exactly; global ids (40,20), (30,20), (10,20): (10,20) wins
    assert sorted(pos) == [2, 3]


@pytest.mark.parametrize("d,rung,grammar,N", [(3, 1, 0, 40), (4, 2, 0, 30), (2, 3, 0, 20), (3, 3, 1, 25)])
def test_levelwise_scores_equal_per_id_scores(orc, d, rung, grammar, N):
    """The whole-space scoring the SIS step uses (phi_{rung-1} evaluated once, new features
    built from stored operands in canonical id order) gives the per-id path's scores and
    validity bit for bit, with every operator of the table enabled and domain errors in
    the data.  The per-id path is itself pinned against numpy above."""
    rng = np.random.default_rng(100 * d + rung)
    X = rng.uniform(-0.5, 3.0, size=(N, d))
    y = rng.normal(size=N)
    sp = orc.Space(d, (1 << 12) - 1, rung, grammar)
    a, va = sp.scores(X, y)
    b, vb = sp.scores_all(X, y)
    assert np.array_equal(va, vb)
    assert np.array_equal(a, b)
    assert 0 < va.sum() < va.size
