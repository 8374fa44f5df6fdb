"""Whitened fits on the GPU (§2.4: W = Sigma^-1/2, SISSO on W y and W Phi) against the
oracle's whitened fit: the ids accepted by SIS at every step and every descriptor equal,
coefficients and RMSE within 1e-6 relative (the FP64 forms' bar)."""
import numpy as np
import pytest

from paper_2410_01752_gb300 import PREC_FP64

pytestmark = pytest.mark.gpu

ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def _whitener(N, kind, rho=0.6, sd=0.3):
    i = np.arange(N)
    Sig = sd ** 2 * rho ** np.abs(i[:, None] - i[None, :])
    if kind == "tri":
        return np.linalg.inv(np.linalg.cholesky(Sig)), Sig
    w, V = np.linalg.eigh(Sig)
    return V @ np.diag(w ** -0.5) @ V.T, Sig


def _problem(seed, N, d):
    rng = np.random.default_rng(seed)
    X = rng.uniform(1, 5, size=(N, d))
    W, Sig = _whitener(N, "sym")
    y = 2 * X[:, 0] * X[:, 1] / X[:, 2 % d] + np.sqrt(X[:, -1]) + np.linalg.cholesky(Sig) @ rng.normal(size=N)
    return X, y


def _compare(c, got, ref, y):
    assert len(got) == len(ref.dims)
    for t, (g, r) in enumerate(zip(got, ref.dims)):
        assert c.sis(t + 1) == ref.sis[t], f"SIS step {t + 1}"
        assert g.ids == r.ids
        np.testing.assert_allclose(g.coef, r.coef, rtol=1e-6, atol=1e-9 * np.abs(y).max())
        assert g.rmse == pytest.approx(r.rmse, rel=1e-6)


@pytest.mark.parametrize("kind", ["sym", "tri"])
@pytest.mark.parametrize("seed,N,d,rung,k,D", [(0, 60, 4, 2, 10, 3), (1, 150, 3, 2, 15, 3), (2, 40, 2, 3, 8, 2)])
def test_whitened_fit_matches_oracle(S, orc, kind, seed, N, d, rung, k, D):
    X, y = _problem(seed, N, d)
    W, _ = _whitener(N, kind)
    m = _mask(orc, ALL9)
    ref = orc.fit(X, y, orc.Space(d, m, rung), k, D, W=W)
    with S.Sisso(X, y, m, rung, k, D, precision=PREC_FP64, whiten=W) as c:
        got = c.fit()
        _compare(c, got, ref, y)


def test_whitened_fit_in_chunks(S, orc):
    """1200 samples and 16 205 candidates: the row-by-row scoring runs in two chunks."""
    X, y = _problem(3, 1200, 5)
    W, _ = _whitener(1200, "tri")
    m = _mask(orc, ALL9)
    ref = orc.fit(X, y, orc.Space(5, m, 2), 10, 2, W=W)
    with S.Sisso(X, y, m, 2, 10, 2, precision=PREC_FP64, whiten=W) as c:
        got = c.fit()
        _compare(c, got, ref, y)


def test_identity_whitening_is_the_plain_fit(S, orc):
    X, y = _problem(4, 80, 4)
    m = _mask(orc, ALL9)
    with S.Sisso(X, y, m, 2, 10, 3, precision=PREC_FP64) as c:
        plain = c.fit()
        sis_plain = [c.sis(t + 1) for t in range(len(plain))]
    with S.Sisso(X, y, m, 2, 10, 3, precision=PREC_FP64, whiten=np.eye(80)) as c:
        white = c.fit()
        assert [c.sis(t + 1) for t in range(len(white))] == sis_plain
    assert [g.ids for g in white] == [g.ids for g in plain]
    for a, b in zip(white, plain):
        np.testing.assert_allclose(a.coef, b.coef, rtol=1e-10)


def test_whitened_fit_with_units_threshold_and_nxp(S, orc):
    """Whitening together with dimensional analysis (x1, x2 one unit, x3 dimensionless),
    the threshold variant of SIS and the NEW_X_PREV grammar at rung 3."""
    X, y = _problem(9, 50, 3)
    W, _ = _whitener(50, "tri")
    labels = [0, 0, -1]
    m = _mask(orc, ALL9)
    sp = orc.Space(3, m, 3, orc.GRAMMAR_NEW_X_PREV, units=labels)
    ref = orc.fit(X, y, sp, 8, 2, sis_threshold=0.3, W=W)
    with S.Sisso(X, y, m, 3, 8, 2, precision=PREC_FP64, grammar=S.GRAMMAR_NEW_X_PREV, units=labels,
                 sis_threshold=0.3, whiten=W) as c:
        got = c.fit()
        _compare(c, got, ref, y)
