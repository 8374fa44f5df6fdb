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
