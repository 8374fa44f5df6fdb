"""GPU parity at the benchmark workloads' full sizes: the CUDA path through the C ABI against
the FP64 oracle's stored fits (tests/golden/*_oracle.json, written by
tests/golden/make_fit_oracle.py from the oracle alone).

Bars: the ids accepted by SIS at every step (§2.2 Eqs. 5-6, in acceptance order) and every
descriptor (§2.3 Eqs. 7-8) bit-exact; coefficients and RMSE within 1e-6 relative for the
FP32 and FP64 forms and 1e-4 relative for the mixed-precision forms (the tolerance stated
for them after the FP64 refit); R^2 within 1e-9 absolute.
"""
import json
import os

import numpy as np
import pytest

from paper_2410_01752_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _golden(name):
    path = os.path.join(HERE, f"{name}_oracle.json")
    if not os.path.exists(path):
        pytest.skip(f"{name}: golden file not written")
    return json.load(open(path))


def _problem(rec):
    P = getattr(inputs, rec["generator"])(rec["p"], **rec["kwargs"])
    assert (P.X.shape[0], P.d, P.rung, P.sis_size, P.max_dim, P.grammar) == (
        rec["N"], rec["d"], rec["rung"], rec["sis_size"], rec["max_dim"], rec["grammar"])
    return P


def _check(c, rec, y, rtol):
    got = c.fit()
    assert len(got) == len(rec["dims"])
    for t, (g, r) in enumerate(zip(got, rec["dims"])):
        assert c.sis(t + 1) == rec["sis"][t], f"SIS step {t + 1}"
        assert g.ids == r["ids"], f"descriptor of dimension {t + 1}"
        np.testing.assert_allclose(g.coef, r["coef"], rtol=rtol, atol=1e-9 * np.abs(y).max())
        assert abs(g.rmse - r["rmse"]) <= rtol * r["rmse"] + 1e-9 * y.std()
        assert g.r2 == pytest.approx(r["r2"], abs=1e-9)
    return got


@pytest.mark.parametrize("name,prec", [("workload2", 1), ("workload2_d6", 1), ("workload2_d6", 0), ("workload2", 2),
                                       ("workload2", 3)])
def test_rung3_fit_full_size(S, name, prec):
    """The benchmark's fit: N=1000, lognormal primaries, rung 3 (2.9e8 candidates at d=10),
    k=100, D<=4 (C(400,4) = 1.05e9 subsets at the last step); plain FP32 and FP64, and the
    mixed BF16 / FP16 forms (tensor-core screening and Gram, FP64 refits)."""
    rec = _golden(name)[0]
    P = _problem(rec)
    with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=prec, grammar=P.grammar,
                 screen=S.SCREEN_TENSOR) as c:
        _check(c, rec, P.y, 1e-6 if prec < 2 else 1e-4)
        st = c.stats()
    if prec < 2:
        assert st["subsets_fit"] == sum(d["subsets"] for d in rec["dims"])
    else:       # the mixed forms with tensor-core screening of the phi_1 x new_2 pairs (on request)
        assert st["screen_tc"] == 1


@pytest.mark.parametrize("prec,rtol,gram", [(1, 1e-6, 0), (1, 1e-6, 2), (2, 1e-4, 0), (3, 1e-4, 0)])
def test_collinear_fit_full_size(S, prec, rtol, gram):
    """The mixed-precision workload at full size: N=65536, six primaries correlated 0.999,
    rung 2, k=200, D<=3 -- plain FP32 (FP64 Gram rows, or the 3xTF32 tensor-core Gram with
    the FP64 refit of the best subsets) and the BF16 / FP16 tensor-core forms."""
    rec = _golden("workload3")[0]
    P = _problem(rec)
    with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=prec, grammar=P.grammar,
                 gram=gram) as c:
        _check(c, rec, P.y, rtol)


def test_rung3_fit_full_size_tf32x3_gram(S):
    """The benchmark's fit (N=1000, d=10, rung 3, k=100, D<=4) in FP32 with the 3xTF32
    tensor-core Gram: the oracle's stored subspaces and descriptors."""
    rec = _golden("workload2")[0]
    P = _problem(rec)
    with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=1, grammar=P.grammar,
                 gram=S.GRAM_TF32X3) as c:
        _check(c, rec, P.y, 1e-6)


def test_d5_fit_full_size(S):
    """The learned proposal's workload, searched exhaustively: rung 2, k=60, D<=5 (C(300,5) =
    1.96e10 subsets at the last step), every stored held-out problem."""
    recs = _golden("workload4")
    for rec in recs:
        P = _problem(rec)
        with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=1, grammar=P.grammar) as c:
            _check(c, rec, P.y, 1e-6)


def test_d5_learned_fit_full_size(S):
    """The fit with the learned proposal at its D = 5 step (a network that returns the
    greedy-completion base score, i.e. the proposal without training) and the certificate:
    every stored held-out problem's descriptors equal the oracle's."""
    recs = _golden("workload4")
    net = S.MLP(0)
    net.set_params(np.zeros(S.MLP_PARAMS, dtype=np.float32))
    for rec in recs:
        P = _problem(rec)
        with S.Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=1, grammar=P.grammar) as c:
            c.set_proposal(net, 0.01)
            _check(c, rec, P.y, 1e-6)
            assert c.stats()["certified_prefixes"] > 0
    net.close()
