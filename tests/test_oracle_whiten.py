"""Pins for the oracle's whitened fit (§2.4: W = Sigma^-1/2, SISSO on W y and W Phi).

Checked against the numpy brute-force iteration with the same transformation, for a
symmetric W (Sigma^-1/2 of an AR(1) noise covariance) and a lower-triangular one (the
inverse Cholesky factor, which also whitens and catches a transposed product); W = I gives
the plain fit; a permutation W gives the plain fit of the permuted samples.
"""
import numpy as np
import pytest

import brute

NAMES = ["+", "-", "*", "/", "sqrt", "^2"]


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def _ar1_cov(N, rho, sd):
    i = np.arange(N)
    return sd ** 2 * rho ** np.abs(i[:, None] - i[None, :])


def _whiteners(S):
    w, V = np.linalg.eigh(S)
    sym = V @ np.diag(w ** -0.5) @ V.T                 # Sigma^-1/2
    tri = np.linalg.inv(np.linalg.cholesky(S))         # L^-1 with Sigma = L L^T
    return {"sym": sym, "tri": tri}


def _problem(seed, N=24):
    rng = np.random.default_rng(seed)
    X = rng.uniform(1, 5, size=(N, 3))
    S = _ar1_cov(N, 0.6, 0.3)
    noise = np.linalg.cholesky(S) @ rng.normal(size=N)
    y = 2 * X[:, 0] / X[:, 1] + np.sqrt(X[:, 2]) + noise
    return X, y, S


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("kind", ["sym", "tri"])
def test_whitened_fit_matches_brute_force(orc, seed, kind):
    X, y, S = _problem(seed)
    W = _whiteners(S)[kind]
    ref = brute.sisso(X, y, 3, NAMES, 2, 4, 3, W=W)
    res = orc.fit(X, y, orc.Space(3, _mask(orc, NAMES), 2), 4, 3, W=W)
    assert len(res.dims) == len(ref)
    for t, (tup, c, rmse, Sacc) in enumerate(ref):
        assert res.dims[t].ids == tup
        assert np.allclose(res.dims[t].coef, c, rtol=1e-8, atol=1e-10)
        assert res.dims[t].rmse == pytest.approx(rmse, rel=1e-8)
        assert sum(res.sis[: t + 1], []) == Sacc


def test_identity_whitening_is_the_plain_fit(orc):
    X, y, _ = _problem(5)
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    a = orc.fit(X, y, sp, 4, 3)
    b = orc.fit(X, y, sp, 4, 3, W=np.eye(len(y)))
    assert a.sis == b.sis
    assert [d.ids for d in a.dims] == [d.ids for d in b.dims]
    for da, db in zip(a.dims, b.dims):
        assert da.coef == db.coef and da.rmse == db.rmse


def test_permutation_whitening_is_the_permuted_fit(orc):
    """W = P (a permutation) maps the samples to a new order: the same subspaces and
    descriptors as the plain fit of the permuted samples, coefficients to rounding."""
    X, y, _ = _problem(6)
    perm = np.random.default_rng(7).permutation(len(y))
    P = np.eye(len(y))[perm]
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    a = orc.fit(X[perm], y[perm], sp, 4, 3)
    b = orc.fit(X, y, sp, 4, 3, W=P)
    assert a.sis == b.sis
    assert [d.ids for d in a.dims] == [d.ids for d in b.dims]
    for da, db in zip(a.dims, b.dims):
        np.testing.assert_allclose(db.coef, da.coef, rtol=1e-10, atol=1e-12)
        assert db.rmse == pytest.approx(da.rmse, rel=1e-10)


def test_whitening_changes_the_fit(orc):
    """With correlated noise the whitened fit is a different least-squares problem: its
    coefficients differ from the plain fit's (the transformation is not a no-op)."""
    X, y, S = _problem(8)
    W = _whiteners(S)["sym"]
    sp = orc.Space(3, _mask(orc, NAMES), 2)
    a = orc.fit(X, y, sp, 4, 1)
    b = orc.fit(X, y, sp, 4, 1, W=W)
    assert not np.allclose(a.dims[0].coef, b.dims[0].coef, rtol=1e-6)


def test_ar1_whitener_whitens_its_covariance():
    """The benchmark's whitening matrix (inputs.ar1_whitener, the Prais-Winsten transform)
    satisfies W Sigma W^T = I for the stationary AR(1) covariance it is built for."""
    from paper_2410_01752_gb300 import inputs
    N, rho, sd = 200, 0.6, 0.05
    i = np.arange(N)
    Sig = sd ** 2 / (1 - rho ** 2) * rho ** np.abs(i[:, None] - i[None, :])
    W = inputs.ar1_whitener(N, rho, sd)
    assert np.abs(W @ Sig @ W.T - np.eye(N)).max() < 1e-12
