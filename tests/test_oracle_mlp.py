"""Pins of the numpy reference network (CPU): analytic gradients against central finite
differences, the bfloat16 rounding against its definition, and the loss of a network
whose output is known in closed form."""
import numpy as np

from oracle import mlp


def _net(seed=0, scale=0.3):
    r = np.random.default_rng(seed)
    p = r.normal(0, scale, mlp.N_PARAMS)
    X = r.normal(size=(16, mlp.N_IN))
    t = r.normal(size=16)
    return p, X, t


def test_gradient_matches_finite_differences():
    p, X, t = _net(1)
    _, g = mlp.loss_and_grad(p, X, t)
    r = np.random.default_rng(2)
    # parameters of every block: W1, b1, W2, b2, w3, b3
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SIZES])
    idx = np.concatenate([r.integers(offs[k], offs[k + 1], 6) for k in range(len(mlp.SIZES))])
    num = mlp.numeric_grad(p, X, t, idx)
    np.testing.assert_allclose(g[idx], num, rtol=1e-5, atol=1e-8)


def test_bf16_rounding():
    # 8 significant bits: the spacing above 1 is 2^-7
    v = np.array([1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0])
    got = mlp.bf16(v)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1; 1 + 3*2^-8 -> 1 + 2^-6
    np.testing.assert_array_equal(got, [1.0, 1.0 + 2 ** -7, 1.0, 1.0 + 2 ** -6, -2.5, 0.0])
    rel = np.abs(mlp.bf16(np.linspace(0.1, 10, 1000)) / np.linspace(0.1, 10, 1000) - 1)
    assert rel.max() <= 2 ** -8


def test_closed_form_network():
    # W1 = 0 except an identity block on the first 20 units, W2 = identity, w3 = 1:
    # y = sum(relu(x)) + b3
    P = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    P["W1"][:mlp.N_IN, :] = np.eye(mlp.N_IN)
    P["W2"] = np.eye(mlp.N_HID)
    P["w3"][:] = 1.0
    P["b3"][0] = 0.5
    X = np.random.default_rng(4).normal(size=(8, mlp.N_IN))
    y, _ = mlp.forward(mlp.pack(P), X)
    np.testing.assert_allclose(y, np.maximum(X, 0).sum(1) + 0.5, rtol=1e-14)
    loss, _ = mlp.loss_and_grad(mlp.pack(P), X, y)
    assert loss == 0.0
