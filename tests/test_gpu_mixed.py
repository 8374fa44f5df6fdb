"""Mixed-precision form: the tensor-core (tcgen05) subspace Gram against an FP64 Gram."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _rows(seed, n, N, collinear=True):
    r = np.random.default_rng(seed)
    X = r.normal(size=(n, N)) + 0.5 * r.normal(size=(1, N))
    if collinear:
        X[1] = X[0] + 0.03 * r.normal(size=N)
    Z = (X - X.mean(1, keepdims=True)) / X.std(1, keepdims=True)
    y = Z[:3].T @ np.array([1.0, -2.0, 0.5]) + 0.1 * r.normal(size=N) + 7.0
    yc = y - y.mean()
    return Z, yc, float(yc.std())


@pytest.mark.parametrize("kind,rel", [(2, 2.0 ** -7), (3, 2.0 ** -10)])
@pytest.mark.parametrize("n,N", [(5, 64), (150, 3000), (301, 20000), (129, 130)])
def test_gram_tc_matches_fp64(S, kind, rel, n, N):
    """Every entry of Z Z^T / N and Z y~ / N within the 16-bit input rounding of the FP64
    product (tiles of 128 rows, ragged edges, split over samples)."""
    Z, yc, sdy = _rows(n + N, n, N)
    G, b = S.gram_tc(Z, yc, sdy, kind)
    G64 = Z @ Z.T / N
    b64 = Z @ yc / N
    assert np.abs(G - G64).max() <= 2 * rel
    assert np.abs(b - b64).max() <= 2 * rel * sdy
    # the diagonal of standardised rows is 1 up to the input rounding
    assert np.abs(np.diag(G) - 1).max() <= 2 * rel


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("seed,N", [(0, 700), (1, 2500)])
def test_fit_mixed_matches_oracle(S, orc, kind, seed, N):
    """The mixed-precision fit (tensor-core Gram, FP64 refit of the 100 best subsets and of
    ill-conditioned ones) on collinear data: the same screened subspaces and descriptors as
    the FP64 oracle, coefficients and RMSE within 1e-4 relative."""
    from paper_2410_01752_gb300 import inputs
    P = inputs.workload3(seed, N=N, sis_size=25, max_dim=3)
    sp = orc.Space(12, P.op_set, 2)
    ref = orc.fit(P.X, P.y, sp, 25, 3)
    with S.Sisso(P.X, P.y, P.op_set, 2, 25, 3, precision=kind) as c:
        got = c.fit()
        for t, (g, r) in enumerate(zip(got, ref.dims)):
            assert c.sis(t + 1) == ref.sis[t]
            assert g.ids == r.ids
            np.testing.assert_allclose(g.coef, r.coef, rtol=1e-4, atol=1e-9 * np.abs(P.y).max())
            assert g.rmse == pytest.approx(r.rmse, rel=1e-4)
    assert len(got) == len(ref.dims)


def test_fit_mixed_equals_plain(S):
    """Mixed and plain FP32 forms reach the same descriptor at equal RMSE (1e-5 relative)."""
    from paper_2410_01752_gb300 import inputs
    P = inputs.workload3(3, N=4096, sis_size=40, max_dim=3)
    with S.Sisso(P.X, P.y, P.op_set, 2, 40, 3, precision=1) as c:
        plain = c.fit()
    for kind in (2, 3):
        with S.Sisso(P.X, P.y, P.op_set, 2, 40, 3, precision=kind) as c:
            mixed = c.fit()
        assert [d.ids for d in mixed] == [d.ids for d in plain]
        for a, b in zip(mixed, plain):
            assert a.rmse == pytest.approx(b.rmse, rel=1e-5)
