"""Contexts created one after another reuse the library's device memory pool: the same results
on every cycle, and the kept memory can be handed back (sisso_release_memory)."""
import numpy as np
import pytest

from paper_2410_01752_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def test_contexts_reuse_pooled_memory(S):
    P = inputs.workload2(0, N=400, d=6)
    runs = []
    for cycle in range(3):
        with S.Sisso(P.X, P.y, P.op_set, P.rung, 20, 3, grammar=P.grammar) as c:
            d = c.fit()
            runs.append(([g.ids for g in d], [g.coef for g in d], [c.sis(t + 1) for t in range(len(d))]))
        if cycle == 1:
            S.release_memory(0)          # the next context maps its buffers afresh
    for ids, coef, sis in runs[1:]:
        assert ids == runs[0][0] and sis == runs[0][2]
        for a, b in zip(coef, runs[0][1]):
            np.testing.assert_array_equal(a, b)
