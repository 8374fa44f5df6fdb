"""Tensor-core (tcgen05) subspace Gram against an FP64 Gram: the mixed forms' 16-bit one and
the FP32 precision's 3xTF32 one; mixed fits against the oracle."""
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


# 3xTF32: the split's error 3 2^-22 plus the FP32 accumulation of a 512-sample run, at most
# about one unit in the last place per MMA: 192 MMAs x 2^-23 (scale: sum |z_i z_j| / N <= 1)
TF32X3_BOUND = 3 * 2.0 ** -22 + 192 * 2.0 ** -23


@pytest.mark.parametrize("kind,tol", [(2, 2.0 ** -6), (3, 2.0 ** -9), (1, TF32X3_BOUND)])
@pytest.mark.parametrize("n,N", [(5, 64), (150, 3000), (301, 20000), (129, 130), (400, 1000)])
def test_gram_tc_matches_fp64(S, kind, tol, n, N):
    """Every entry of Z Z^T / N and Z y~ / N within the error bound of its form (tiles of 128
    rows, ragged edges, split over samples).  BF16 / FP16 operands: twice their unit
    roundoff.  3xTF32 (kind 1): |z_i z_j - (h_i h_j + h_i l_j + l_i h_j)| <= 3 2^-22 |z_i z_j|
    and sum |z_i z_j| / N <= 1 for standardised rows (Cauchy-Schwarz), plus the tensor
    cores' FP32 accumulation over 512-sample runs: 2.4e-5, which a single TF32 product
    (error up to 2^-11 = 4.9e-4) would miss by far."""
    Z, yc, sdy = _rows(n + N, n, N)
    G, b = S.gram_tc(Z, yc, sdy, kind)
    G64 = Z @ Z.T / N
    b64 = Z @ yc / N
    assert np.abs(G - G64).max() <= tol
    assert np.abs(b - b64).max() <= tol * sdy
    # the diagonal of standardised rows is 1 up to the same error
    assert np.abs(np.diag(G) - 1).max() <= tol


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


@pytest.mark.parametrize("seed,N", [(0, 700), (1, 2500)])
def test_fit_fp32_tf32x3_gram_matches_oracle(S, orc, seed, N):
    """FP32 precision with the 3xTF32 tensor-core Gram (sisso_opts.gram = TF32X3) on
    collinear data: the same screened subspaces and descriptors as the FP64 oracle; the
    winner is refit in FP64 from the standardised rows, so coefficients and RMSE within
    1e-6 relative."""
    from paper_2410_01752_gb300 import inputs
    P = inputs.workload3(seed, N=N, sis_size=25, max_dim=3)
    sp = orc.Space(12, P.op_set, 2)
    ref = orc.fit(P.X, P.y, sp, 25, 3)
    with S.Sisso(P.X, P.y, P.op_set, 2, 25, 3, precision=1, gram=S.GRAM_TF32X3) as c:
        got = c.fit()
        for t, (g, r) in enumerate(zip(got, ref.dims)):
            assert c.sis(t + 1) == ref.sis[t]
            assert g.ids == r.ids
            np.testing.assert_allclose(g.coef, r.coef, rtol=1e-6, atol=1e-9 * np.abs(P.y).max())
            assert g.rmse == pytest.approx(r.rmse, rel=1e-6)
    assert len(got) == len(ref.dims)
