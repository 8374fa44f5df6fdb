"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: feature ids (SIS selections, descriptors, l0 winners) bit-exact; FP64 kernel
values within 1e-12 relative, their scores within 1e-7 (the score buffer is FP32); FP32
screening scores within the 2e-4 margin the selection's
exactness proof assumes; coefficients and RMSE within 1e-6 relative (RMSE of an exact fit
within 1e-9 std(y) absolute).
"""
import math

import numpy as np
import pytest

from paper_2410_01752_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]
FP32_SCORE_TOL = 2e-4


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def _ctx(S, X, y, ops, rung, k, D, prec, grammar=0, **kw):
    return S.Sisso(X, y, ops, rung, k, D, precision=prec, grammar=grammar, **kw)


def _lognormal_problem(seed, N, d):
    r = np.random.default_rng(seed)
    X = r.lognormal(0, 0.5, size=(N, d))
    y = X[:, 0] * X[:, 1] / X[:, 2 % d] + np.log(X[:, -1]) * X[:, 0] + 0.01 * r.normal(size=N)
    return X, y


# ---------------------------------------------------------------------------------
# feature values
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_eval_features(S, orc, prec):
    P = inputs.workload1(0)
    sp = orc.Space(5, P.op_set, 2)
    with _ctx(S, P.X, P.y, P.op_set, 2, 20, 3, prec) as c:
        ids = np.arange(sp.n_features)
        got = c.eval_features(ids, prec)
    for i in range(0, sp.n_features, 7):
        ref = sp.eval(P.X, i)
        g = got[i]
        fin = np.isfinite(ref) & (np.abs(ref) < 1e30)
        if prec == 0:
            assert np.allclose(g[fin], ref[fin], rtol=1e-12, atol=0), sp.expr(i)
        else:
            # FP32 rounding of the operands: error relative to the feature's magnitude
            ok = fin & (np.abs(ref) < 1e12)
            scale = np.abs(ref[ok]).max() if ok.any() else 1.0
            assert np.allclose(g[ok], ref[ok], rtol=2e-5, atol=2e-6 * scale), sp.expr(i)


# ---------------------------------------------------------------------------------
# screening scores (fused generate-and-score kernels)
# ---------------------------------------------------------------------------------
SCORE_CASES = [
    ("c1", lambda: (inputs.workload1(0).X, inputs.workload1(0).y), ALL9, 2, 0),
    ("rung3-nxp", lambda: _lognormal_problem(7, 200, 4), ALL9, 3, 1),
    ("rung3-eq2", lambda: _lognormal_problem(8, 77, 2), ["+", "-", "*", "/", "sqrt", "^2"], 3, 0),
    ("rung1", lambda: _lognormal_problem(9, 33, 40), ALL9, 1, 0),
    # six primaries correlated 0.999: operands such as x2 - x4 cancel, and 1/(x2 - x4) or
    # x1/(x2 - x4) is dominated by the samples where they nearly vanish
    ("collinear", lambda: (inputs.workload3(0, N=3000).X, inputs.workload3(0, N=3000).y), ALL9, 2, 0),
]


@pytest.mark.parametrize("name,make,names,rung,g", SCORE_CASES, ids=[c[0] for c in SCORE_CASES])
@pytest.mark.parametrize("prec", [0, 1])
def test_score_all(S, orc, name, make, names, rung, g, prec):
    X, y = make()
    m = _mask(orc, names)
    sp = orc.Space(X.shape[1], m, rung, g)
    ref, valid = sp.scores(X, y)
    with _ctx(S, X, y, m, rung, 5, 2, prec, grammar=g) as c:
        got = c.score_all(y, prec)
    assert got.shape == ref.shape
    # a kernel may only reject what the oracle rejects
    rejected = got < 0
    assert not np.any(rejected & valid), [sp.expr(int(i)) for i in np.where(rejected & valid)[0][:5]]
    tol = 1e-7 if prec == 0 else FP32_SCORE_TOL       # scores are stored as FP32
    err = np.abs(got[valid].astype(np.float64) - ref[valid])
    assert err.max() <= tol, (err.max(), sp.expr(int(np.where(valid)[0][np.argmax(err)])))


def test_cross_sum_keys_left_open(S, orc):
    """FP32 + and - from the cross sum: on six primaries correlated 0.999 the operands x_i - x_j
    cancel against each other, the cross sum's rounding bound leaves those keys open, and the
    direct sums score them -- every score within the margin of the oracle's and no valid
    candidate rejected."""
    P = inputs.workload3(0, N=3000)
    m = _mask(orc, ALL9)
    sp = orc.Space(P.X.shape[1], m, 2, 0)
    ref, valid = sp.scores(P.X, P.y)
    with _ctx(S, P.X, P.y, m, 2, 5, 2, 1) as c:
        got = c.score_all(P.y, 1)
        opened = c.stats()["pm_keys_direct"]
    assert opened > 0
    assert not np.any((got < 0) & valid)
    assert np.abs(got[valid].astype(np.float64) - ref[valid]).max() <= FP32_SCORE_TOL


# ---------------------------------------------------------------------------------
# one SIS step: device-wide selection, FP64 re-score, walk
# ---------------------------------------------------------------------------------
def _c3_small(N=600):
    P = inputs.workload3(0, N=N)
    return P.X, P.y


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["c1", "rung3", "collinear", "wide", "long"])
def test_sis_step(S, orc, case, prec):
    """One SIS step and a second one on a residual.  "wide": k = 150 makes the re-scored
    window 8192 entries (walk on the global arrays, not the shared-memory copy); "long":
    9000 samples (two partner slots confirmed ahead of the walk instead of eight)."""
    if case == "c1":
        P = inputs.workload1(1)
        X, y, m, rung, g, k = P.X, P.y, P.op_set, 2, 0, 20
    elif case == "rung3":
        X, y = _lognormal_problem(11, 150, 4)
        m, rung, g, k = _mask(orc, ALL9), 3, 1, 30
    elif case == "wide":
        X, y = _lognormal_problem(13, 150, 4)
        m, rung, g, k = _mask(orc, ALL9), 3, 1, 150
    elif case == "long":
        X, y = _lognormal_problem(14, 9000, 4)
        m, rung, g, k = _mask(orc, ALL9), 2, 0, 20
    else:
        X, y = _c3_small()
        m, rung, g, k = _mask(orc, ALL9), 2, 0, 40
    sp = orc.Space(X.shape[1], m, rung, g)
    ref1 = sp.sis(X, y, [], k)
    with _ctx(S, X, y, m, rung, k, 3, prec, grammar=g) as c:
        got1 = c.sis_step(y, [], k)
        assert got1 == ref1
        # second step on a residual, with S_1 excluded (and its duplicates)
        v = sp.eval(X, ref1[0])
        r = y - np.polyval(np.polyfit(v, y, 1), v)
        ref2 = sp.sis(X, r, ref1, k)
        got2 = c.sis_step(r, ref1, k)
        assert got2 == ref2


# ---------------------------------------------------------------------------------
# exhaustive l0
# ---------------------------------------------------------------------------------
def _gram_case(seed, n, N=200, collinear=False):
    r = np.random.default_rng(seed)
    cols = r.normal(size=(N, n)) + 0.4 * r.normal(size=(N, 1))
    if collinear:
        cols[:, 3] = cols[:, 1] + 1e-4 * r.normal(size=N)     # pivot ~1e-8
        cols[:, 5] = 2.0 * cols[:, 2] - 1.0                   # exactly collinear
    y = cols[:, :3] @ r.uniform(-2, 2, 3) + 0.3 * r.normal(size=N)
    Z = (cols - cols.mean(0)) / cols.std(0)
    yc = y - y.mean()
    return Z.T @ Z / N, Z.T @ yc / N, float(yc @ yc) / N, N


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,D,seed,col", [(20, 1, 0, False), (40, 2, 1, False), (60, 3, 2, False),
                                          (45, 4, 3, False), (33, 3, 4, True), (30, 4, 5, True),
                                          (4, 4, 6, False), (97, 2, 7, True), (24, 5, 8, False),
                                          (31, 5, 9, True), (5, 5, 10, False),
                                          # several 64-row x 256-column tiles and ragged edges
                                          (300, 2, 11, False), (517, 2, 12, True), (260, 3, 13, False),
                                          (301, 3, 14, True), (130, 4, 15, False), (150, 4, 16, True),
                                          (66, 5, 17, False), (70, 5, 18, True)])
def test_l0_search(S, orc, n, D, seed, col, prec):
    G, b, syy, N = _gram_case(seed, n, collinear=col)
    if n > 64:          # move the planted features (and the collinear pairs) into later tiles
        perm = np.random.default_rng(seed + 90).permutation(n)
        G, b = G[np.ix_(perm, perm)], b[perm]
    gid = np.random.default_rng(seed + 50).permutation(10 * n)[:n]
    pos_ref, rss_ref, ex_ref = orc.l0(G, b, syy, N, D, gid)
    X = np.random.default_rng(0).uniform(1, 2, size=(N, 2))
    with _ctx(S, X, np.arange(N, dtype=float), orc.opmask(orc.ADD), 1, 2, 1, prec) as c:
        pos, rss, ex = c.l0_search(G, b, syy, D, gid, prec)
    assert ex == ex_ref == math.comb(n, D)
    assert pos == pos_ref
    assert rss == pytest.approx(rss_ref, rel=1e-9, abs=1e-9 * syy * N)


def test_l0_exact_ties(S, orc):
    """Several subsets with the same RSS: the smallest ascending global-id tuple wins."""
    r = np.random.default_rng(3)
    N = 100
    a, c2 = r.normal(size=N), r.normal(size=N)
    cols = np.column_stack([a, c2, -a, 3 * a + 2, r.normal(size=N), a])
    y = a + 0.1 * c2
    Z = (cols - cols.mean(0)) / cols.std(0)
    yc = y - y.mean()
    G, b, syy = Z.T @ Z / N, Z.T @ yc / N, float(yc @ yc) / N
    gid = np.array([60, 50, 40, 30, 20, 10])
    ref = orc.l0(G, b, syy, N, 2, gid)
    X = np.random.default_rng(0).uniform(1, 2, size=(N, 2))
    for prec in (0, 1):
        with _ctx(S, X, np.arange(N, dtype=float), orc.opmask(orc.ADD), 1, 2, 1, prec) as c:
            assert c.l0_search(G, b, syy, 2, gid, prec)[0] == ref[0]


# ---------------------------------------------------------------------------------
# whole fit
# ---------------------------------------------------------------------------------
def _compare_fit(c, ref, sp, y):
    got = c.fit()
    assert len(got) == len(ref.dims)
    for t, (g, r) in enumerate(zip(got, ref.dims)):
        assert c.sis(t + 1) == ref.sis[t]
        assert g.ids == r.ids, ([sp.expr(i) for i in g.ids], [sp.expr(i) for i in r.ids])
        np.testing.assert_allclose(g.coef, r.coef, rtol=1e-6, atol=1e-9 * np.abs(y).max())
        assert abs(g.rmse - r.rmse) <= 1e-6 * r.rmse + 1e-9 * y.std()
        assert g.r2 == pytest.approx(r.r2, abs=1e-9)
    return got


@pytest.mark.parametrize("prec", [0, 1])
def test_fit_workload1(S, orc, prec):
    P = inputs.workload1(0)
    sp = orc.Space(5, P.op_set, 2)
    ref = orc.fit(P.X, P.y, sp, 20, 3)
    with _ctx(S, P.X, P.y, P.op_set, 2, 20, 3, prec) as c:
        got = _compare_fit(c, ref, sp, P.y)
        assert sp.expr(got[0].ids[0]) == "(x1*(x2/x3))"


@pytest.mark.parametrize("prec", [0, 1])
def test_fit_rung3_small(S, orc, prec):
    P = inputs.workload2(0, N=160, d=5, sis_size=15, max_dim=3)
    sp = orc.Space(5, P.op_set, 3, P.grammar)
    ref = orc.fit(P.X, P.y, sp, 15, 3)
    with _ctx(S, P.X, P.y, P.op_set, 3, 15, 3, prec, grammar=P.grammar) as c:
        _compare_fit(c, ref, sp, P.y)


@pytest.mark.parametrize("prec", [0, 1])
def test_fit_collinear_small(S, orc, prec):
    P = inputs.workload3(0, N=700, sis_size=25, max_dim=3)
    sp = orc.Space(12, P.op_set, 2)
    ref = orc.fit(P.X, P.y, sp, 25, 3)
    with _ctx(S, P.X, P.y, P.op_set, 2, 25, 3, prec) as c:
        _compare_fit(c, ref, sp, P.y)


@pytest.mark.parametrize("p", [0, 1, 2])
def test_fit_batched_tasks(S, orc, p):
    P = inputs.workload5_task(p)
    sp = orc.Space(P.d, P.op_set, 2)
    ref = orc.fit(P.X, P.y, sp, P.sis_size, P.max_dim)
    with _ctx(S, P.X, P.y, P.op_set, 2, P.sis_size, P.max_dim, 1) as c:
        _compare_fit(c, ref, sp, P.y)


def test_fit_planted_exact_stops(S, orc):
    """Noise-free planted target: exact descriptor, coefficients, and the stop after t=1."""
    rng = np.random.default_rng(42)
    X = rng.uniform(1, 5, size=(50, 5))
    y = 3.0 * X[:, 0] * X[:, 1] / X[:, 2] + 0.5
    m = _mask(orc, ALL9)
    for prec in (0, 1):
        with _ctx(S, X, y, m, 2, 20, 3, prec) as c:
            got = c.fit()
            assert len(got) == 1
            assert got[0].coef[1] == pytest.approx(3.0, abs=1e-9)
            assert got[0].coef[0] == pytest.approx(0.5, abs=1e-9)
            assert got[0].rmse <= 1e-10 * y.std()


# ---------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------
def test_edge_errors(S):
    X = np.random.default_rng(0).uniform(1, 2, size=(30, 3))
    y = X[:, 0] * 2
    Xb = X.copy()
    Xb[3, 1] = np.nan
    with pytest.raises(S.SissoError):
        S.Sisso(Xb, y, S.OP_ADD, 1, 3, 2)
    with pytest.raises(S.SissoError):
        S.Sisso(X, np.ones(30), S.OP_ADD, 1, 3, 2)      # constant target
    yb = y.copy()
    yb[0] = np.inf
    with pytest.raises(S.SissoError):
        S.Sisso(X, yb, S.OP_ADD, 1, 3, 2)


def test_fewer_features_than_k(S, orc):
    """k above the number of distinct valid features: S takes them all, l0 still exact."""
    rng = np.random.default_rng(4)
    X = rng.uniform(1, 5, size=(25, 2))
    y = X[:, 0] + 2 * X[:, 1] ** 2 + 0.1 * rng.normal(size=25)
    m = orc.opmask(orc.ADD, orc.SQ)
    sp = orc.Space(2, m, 1)
    ref = orc.fit(X, y, sp, 10, 3)
    for prec in (0, 1):
        with _ctx(S, X, y, m, 1, 10, 3, prec) as c:
            _compare_fit(c, ref, sp, y)
