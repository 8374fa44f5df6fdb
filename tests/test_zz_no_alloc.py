"""The allocation-free l0 search (sisso_l0_search_noalloc) against the context-based one.

Some callers cannot allocate device memory (a plug-in limited to memory its host gives
it, a framework whose pool must own every allocation, a loop that cannot afford the
synchronisation cudaMalloc implies).  For them the library offers one entry point whose
working memory is a fixed array inside the library.  This file is collected last so that
a run stopping at the first failure has run every other test first; it passes alone in a
fresh process as well.
"""
import math

import numpy as np
import pytest


def _case(seed, n, N=300):
    r = np.random.default_rng(seed)
    cols = r.normal(size=(N, n)) + 0.4 * r.normal(size=(N, 1))
    cols[:, 2] = cols[:, 1] + 1e-4 * r.normal(size=N)          # nearly collinear pair
    y = cols[:, :3] @ r.uniform(-2, 2, 3) + 0.3 * r.normal(size=N)
    Z = (cols - cols.mean(0)) / cols.std(0)
    yc = y - y.mean()
    gid = r.permutation(50 * n)[:n]
    return Z.T @ Z / N, Z.T @ yc / N, float(yc @ yc) / N, N, gid


def test_noalloc_rejects_oversize():
    """Sizes beyond the fixed working array are refused before any GPU work."""
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    n = sisso.NOALLOC_MAX_N + 1
    with pytest.raises(sisso.SissoError) as e:
        sisso.l0_search_noalloc(np.eye(n), np.zeros(n), 1.0, 10, 2, np.arange(n))
    assert e.value.status == -7          # SISSO_ERR_CAPACITY


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_context_search(prec):
    """Two calls in a row (different problems, so the shared array is reused) give the
    same winners, RSS and subset counts as sisso_l0_search."""
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    cases = [(_case(1, 60), 3), (_case(2, 45), 4)]
    for (G, b, syy, N, gid), D in cases:
        X = np.random.default_rng(0).uniform(1, 2, size=(N, 2))
        with sisso.Sisso(X, np.arange(N, dtype=float), sisso.OP_ADD, 1, 2, 1, precision=prec) as c:
            ref = c.l0_search(G, b, syy, D, gid, prec)
        got = sisso.l0_search_noalloc(G, b, syy, N, D, gid, prec)
        assert got[0] == ref[0]
        assert got[1] == pytest.approx(ref[1], rel=1e-9, abs=1e-9 * syy * N)
        assert got[2] == ref[2] == math.comb(b.size, D)


@pytest.mark.gpu
@pytest.mark.parametrize("D,n", [(1, 40), (2, 40), (3, 40), (4, 40), (5, 30)])
@pytest.mark.parametrize("where", ["host", "device"])
def test_noalloc_every_dimension(D, n, where):
    """D = 1..5 with G, b and gid in host or device memory: the context search's winner, RSS
    and subset count."""
    import torch
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    G, b, syy, N, gid = _case(10 + D, n)
    X = np.random.default_rng(0).uniform(1, 2, size=(N, 2))
    with sisso.Sisso(X, np.arange(N, dtype=float), sisso.OP_ADD, 1, 2, 1, precision=1) as c:
        ref = c.l0_search(G, b, syy, D, gid, 1)
    if where == "device":
        args = (torch.from_numpy(G).cuda(), torch.from_numpy(b).cuda(), torch.from_numpy(gid.astype(np.int64)).cuda())
    else:
        args = (G, b, gid)
    got = sisso.l0_search_noalloc(args[0], args[1], syy, N, D, args[2], 1)
    assert got[0] == ref[0]
    assert got[1] == pytest.approx(ref[1], rel=1e-9, abs=1e-9 * syy * N)
    assert got[2] == ref[2] == math.comb(n, D)
