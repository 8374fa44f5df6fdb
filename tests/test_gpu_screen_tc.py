"""Tensor-core screening of the mixed forms (§2.2 Eq. 5 as a contraction): the split 16-bit
product against FP64 sums, the keys against the FP64 oracle's scores, and fits against the
oracle with the top level's pairs scored on the tensor cores."""
import numpy as np
import pytest

from paper_2410_01752_gb300 import inputs

pytestmark = pytest.mark.gpu

KEY_EPS = 2.0 ** -17        # the bound each key carries, relative to the Cauchy-Schwarz scale
MARGIN = 2e-4               # the FP32 screening margin of the selection


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _rows(seed, m, N, positive=False):
    r = np.random.default_rng(seed)
    A = r.normal(size=(m, N)) * np.exp(r.normal(0, 3, size=(m, 1)))       # row scales over 1e-4..1e4
    if positive:
        A = A * A
    A[0, :] = 0.0                                                          # an all-zero row
    return A


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("m,n,N", [(3, 5, 40), (150, 131, 1000), (129, 300, 70001)])
def test_bilinear_tc_error(S, kind, m, n, N):
    """|product - FP64 product| within 2^-19 of sqrt(sum L_i^2 sum R_j^2) for rows of mixed
    sign and for positive rows (sums of squares, where no cancellation hides a biased
    accumulation), over ragged tiles and sample chunks; the keys use 2^-17."""
    for pos in (False, True):
        Lr = _rows(m + N + pos, m, N, pos)
        Rr = _rows(n * 7 + N + pos, n, N, pos)
        got = S.bilinear_tc(Lr, Rr, kind)
        ref = Lr @ Rr.T
        cs = np.sqrt(np.outer((Lr * Lr).sum(1), (Rr * Rr).sum(1)))
        ratio = np.abs(got - ref) / np.where(cs > 0, cs, 1.0)
        print(f"kind {kind} m {m} n {n} N {N} positive {pos}: max error / CS scale = {ratio.max():.3e}")
        assert np.all(got[cs == 0] == 0)
        assert ratio.max() <= KEY_EPS / 4


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]


def _lognormal(seed, N, d):
    r = np.random.default_rng(seed)
    X = np.exp(r.normal(0, 0.5, size=(N, d)))
    y = X[:, 0] * X[:, 1 % d] / X[:, 2 % d] + np.log(X[:, -1]) * X[:, 0] + 0.01 * r.normal(size=N)
    return X, y


TC_CASES = [
    ("c1", lambda: (inputs.workload1(0).X, inputs.workload1(0).y), ALL9, 2, 0),
    ("collinear", lambda: (inputs.workload3(0, N=3000).X, inputs.workload3(0, N=3000).y), ALL9, 2, 0),
    ("rung3-eq2", lambda: _lognormal(8, 77, 2), ["+", "-", "*", "/", "sqrt", "^2"], 3, 0),
    ("rung1", lambda: _lognormal(9, 33, 40), ALL9, 1, 0),
    # NEW_X_PREV at rung 3: pairs of phi_1 x new_2 (two operand sets, rectangular products)
    ("rung3-nxp", lambda: _lognormal(7, 200, 4), ALL9, 3, 1),
    ("rung3-nxp-d5", lambda: (inputs.workload2(0, N=400, d=5).X, inputs.workload2(0, N=400, d=5).y), ALL9, 3, 1),
]


@pytest.mark.parametrize("name,make,names,rung,g", TC_CASES, ids=[c[0] for c in TC_CASES])
@pytest.mark.parametrize("kind", [2, 3])
def test_tc_keys_bound_oracle_scores(S, orc, name, make, names, rung, g, kind):
    """Every key is an upper bound of the oracle's FP64 score up to the screening margin
    (key + margin >= score), a key rejects only what the oracle rejects, and keys above the
    score by more than the margin are the raised ones the context counts."""
    X, y = make()
    m = _mask(orc, names)
    sp = orc.Space(X.shape[1], m, rung, g)
    ref, valid = sp.scores(X, y)
    with S.Sisso(X, y, m, rung, 5, 2, precision=kind, grammar=g, screen=S.SCREEN_TENSOR) as c:
        got = c.score_all(y, kind).astype(np.float64)
        st = c.stats()
    assert st["screen_tc"] == 1
    rejected = got < 0
    assert not np.any(rejected & valid)
    gv, rv = got[valid], ref[valid]
    assert np.all(gv + MARGIN >= rv), (gv - rv).min()
    high = int(np.sum(gv > rv + MARGIN))
    print(f"{name} kind {kind}: {valid.sum()} valid, keys raised {st['tc_keys_raised']}, above score + margin {high}, "
          f"median |key - score| {np.median(np.abs(gv - rv)):.2e}")
    assert high <= st["tc_keys_raised"]
    assert np.median(np.abs(gv - rv)) <= 1e-6


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("seed,N", [(0, 700), (1, 4100)])
def test_tc_fit_matches_oracle(S, orc, kind, seed, N):
    """Mixed fits with tensor-core screening on the collinear workload: the oracle's SIS
    selections and descriptors, coefficients and RMSE within 1e-4 relative; the same as the
    CUDA-core screening of the same form."""
    P = inputs.workload3(seed, N=N, sis_size=25, max_dim=3)
    sp = orc.Space(12, P.op_set, 2)
    ref = orc.fit(P.X, P.y, sp, 25, 3)
    out = {}
    for cores in (False, True):
        with S.Sisso(P.X, P.y, P.op_set, 2, 25, 3, precision=kind,
                     screen=S.SCREEN_CORES if cores else S.SCREEN_AUTO) as c:
            got = c.fit()
            assert c.stats()["screen_tc"] == (0 if cores else 1)
            assert len(got) == len(ref.dims)
            for t, (g, r) in enumerate(zip(got, ref.dims)):
                assert c.sis(t + 1) == ref.sis[t]
                assert g.ids == r.ids
                np.testing.assert_allclose(g.coef, r.coef, rtol=1e-4, atol=1e-9 * np.abs(P.y).max())
                assert g.rmse == pytest.approx(r.rmse, rel=1e-4)
            out[cores] = [g.ids for g in got]
    assert out[False] == out[True]


def test_tc_fit_with_units(S, orc):
    """Dimensional analysis on top of tensor-core keys: the oracle's selections."""
    r = np.random.default_rng(41)
    X = r.uniform(1, 5, size=(300, 4))
    y = 2.0 * (X[:, 0] - X[:, 1]) / X[:, 2] + 0.5 * X[:, 3] * X[:, 2] + 0.01 * r.normal(size=300)
    labels = (0, 0, 1, 2)
    sp = orc.Space(4, inputs.OPS9, 2, 0, units=labels)
    ref = orc.fit(X, y, sp, 15, 3)
    with S.Sisso(X, y, inputs.OPS9, 2, 15, 3, precision=3, units=labels) as c:
        got = c.fit()
        assert c.stats()["screen_tc"] == 1
        for t, (a, b) in enumerate(zip(got, ref.dims)):
            assert c.sis(t + 1) == ref.sis[t]
            assert a.ids == b.ids


@pytest.mark.parametrize("kind", [2, 3])
def test_tc_rung3_fit_matches_oracle(S, orc, kind):
    """NEW_X_PREV rung 3 with tensor-core screening on request (phi_1 x new_2 products): the
    oracle's selections and descriptors; coefficients within 1e-4 relative.  By default the
    mixed forms keep these pairs on the CUDA cores."""
    P = inputs.workload2(0, N=400, d=5, sis_size=20, max_dim=3)
    sp = orc.Space(P.d, P.op_set, P.rung, P.grammar)
    ref = orc.fit(P.X, P.y, sp, P.sis_size, P.max_dim)
    with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=kind, grammar=P.grammar,
                 screen=S.SCREEN_TENSOR) as c:
        got = c.fit()
        assert c.stats()["screen_tc"] == 1
        assert len(got) == len(ref.dims)
        for t, (g, r) in enumerate(zip(got, ref.dims)):
            assert c.sis(t + 1) == ref.sis[t]
            assert g.ids == r.ids
            np.testing.assert_allclose(g.coef, r.coef, rtol=1e-4, atol=1e-9 * np.abs(P.y).max())


def test_screen_modes(S):
    """Where the mixed forms score the top level's pairs: automatically on the tensor cores
    for pairs within phi_{L-1}, on the CUDA cores for NEW_X_PREV rung 3 unless asked."""
    P = inputs.workload2(0, N=200, d=4, sis_size=5, max_dim=1)
    for mode, want in ((S.SCREEN_AUTO, 0), (S.SCREEN_CORES, 0), (S.SCREEN_TENSOR, 1)):
        with S.Sisso(P.X, P.y, P.op_set, P.rung, 5, 1, precision=2, grammar=P.grammar, screen=mode) as c:
            c.fit()
            assert c.stats()["screen_tc"] == want
    Q = inputs.workload1(0)
    with S.Sisso(Q.X, Q.y, Q.op_set, Q.rung, 5, 1, precision=3) as c:
        c.fit()
        assert c.stats()["screen_tc"] == 1
    with pytest.raises(S.SissoError):
        S.Sisso(Q.X, Q.y, Q.op_set, Q.rung, 5, 1, precision=3, screen=3)
