"""Pins for the oracle's feature space (§2.1, Eq. 2 and Eq. 3)."""
import itertools
import os

import numpy as np
import pytest

import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example_phi.txt")
ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def _golden():
    levels, bounds = {}, {}
    for line in open(GOLDEN):
        line = line.strip()
        if line.startswith("# bound:"):
            lv, b = line.split(":")[1].split()
            bounds[int(lv)] = int(b)
        elif line and not line.startswith("#"):
            lv, expr = line.split(":", 1)
            levels.setdefault(int(lv), []).append(expr.strip())
    return levels, bounds


def test_worked_example_counts_and_values(orc):
    """§2.1 worked example: |phi_1| = 4, |phi_2| = 14, and the features are exactly the
    paper's (matched one-to-one by their values at random points)."""
    levels, _ = _golden()
    sp = orc.Space(2, orc.opmask(orc.ADD, orc.MUL), 2)
    sizes = sp.sizes()
    assert sizes == [2, len(levels[1]), len(levels[2])] == [2, 4, 14]
    X = np.random.default_rng(0).uniform(1, 5, size=(7, 2))
    x1, x2 = X[:, 0], X[:, 1]
    for lv in (1, 2):
        paper = sorted(tuple(np.round(eval(e, {"x1": x1, "x2": x2}), 9)) for e in levels[lv])
        ours = sorted(tuple(np.round(sp.eval(X, i), 9)) for i in range(sizes[lv]))
        assert paper == ours
    # the 14 level-2 features are pairwise distinct ("14 unique")
    vals = {tuple(np.round(sp.eval(X, i), 9)) for i in range(14)}
    assert len(vals) == 14


def test_worked_example_bound(orc):
    """Eq. 3 with the example's numbers: the bound gives 4 and 16 (identity counted as the
    unary operator, + and x symmetric)."""
    _, bounds = _golden()
    d, m_u, m_bs, m_bns = 2, 1, 2, 0
    d1 = m_u * d + (m_bs / 2 + m_bns) * d * (d - 1)
    d2 = m_u * d1 + (m_bs / 2 + m_bns) * d1 * (d1 - 1)
    assert (d1, d2) == (bounds[1], bounds[2]) == (4, 16)


@pytest.mark.parametrize("d,names,rung", [
    (2, ["+", "*"], 3), (3, ALL9, 2), (5, ALL9, 2), (4, ["+", "-", "/", "exp"], 2),
    (3, ["*", "/", "sqrt", "sin", "^3", "exp-"], 2), (10, ALL9, 2), (12, ALL9, 2)])
def test_count_bound_eq3(orc, d, names, rung):
    """Every level satisfies Eq. 3 (identity counted as one more unary operator; - and /
    counted as non-symmetric as the paper does)."""
    sp = orc.Space(d, _mask(orc, names), rung)
    sizes = sp.sizes()
    m_u = 1 + sum(n in brute.UNARY for n in names)
    m_bs = sum(n in ("+", "*") for n in names)
    m_bns = sum(n in ("-", "/") for n in names)
    for lv in range(1, rung + 1):
        P = sizes[lv - 1]
        assert sizes[lv] <= m_u * P + (m_bs / 2 + m_bns) * P * (P - 1)


@pytest.mark.parametrize("d,names,rung,nxp", [
    (2, ["+", "*"], 3, False), (2, ["+", "*"], 3, True), (3, ALL9, 2, False),
    (2, ["-", "/", "log", "^2"], 3, False), (2, ["-", "/", "log", "^2"], 3, True),
    (3, ["+", "/", "sqrt"], 3, True)])
def test_enumeration_matches_brute_force(orc, d, names, rung, nxp):
    """The oracle's closed-form sections and decode equal an explicit double loop over the
    pair rule, id by id (operator, operands and expression string)."""
    feats, sizes = brute.space(d, names, rung, new_x_prev=nxp)
    sp = orc.Space(d, _mask(orc, names), rung, orc.GRAMMAR_NEW_X_PREV if nxp else orc.GRAMMAR_EQ2)
    assert sp.sizes() == sizes
    for i, f in enumerate(feats):
        assert sp.expr(i) == brute.to_str(f)


def test_pair_predicate_matches_row_ranges(orc):
    """oracle_pair_allowed (the rule as a predicate) agrees with the enumerated sections."""
    for nxp in (0, 1):
        sp = orc.Space(3, _mask(orc, ["+", "-", "*", "/"]), 3, nxp)
        sizes = sp.sizes()
        for lv in (1, 2, 3):
            P, Q = sizes[lv - 1], (sizes[lv - 2] if lv >= 2 else 0)
            for op in range(4):
                n = sum(orc.lib().oracle_pair_allowed(nxp, lv, op, i, j, P, Q)
                        for i in range(P) for j in range(P))
                assert n == sp.section_count(lv, op)


def test_paper_scale_counts(orc):
    """Sizes of the spaces the benchmarks use: d=5 rung 2 (16 205), d=10 rung 2 (203 785),
    d=12 rung 2 (405 027), d=10 rung 3 with one rung-3 operand from phi_1 (2.91e8)."""
    ops = _mask(orc, ALL9)
    assert orc.Space(5, ops, 2).sizes() == [5, 80, 16205]
    assert orc.Space(10, ops, 2).sizes() == [10, 285, 203785]
    assert orc.Space(12, ops, 2).sizes() == [12, 402, 405027]
    assert orc.Space(10, ops, 3, orc.GRAMMAR_NEW_X_PREV).sizes()[-1] == 291208785
    # rung-2 spaces do not depend on the grammar
    assert orc.Space(7, ops, 2, orc.GRAMMAR_NEW_X_PREV).sizes() == orc.Space(7, ops, 2).sizes()


def test_decode_spot_checks_large_space(orc):
    """Decoding ids in the 2.9e8-feature space: children lie at lower levels, in range,
    and the level-3 binary features pair a phi_2-new operand with a phi_1 operand."""
    sp = orc.Space(10, _mask(orc, ALL9), 3, orc.GRAMMAR_NEW_X_PREV)
    sizes = sp.sizes()
    rng = np.random.default_rng(3)
    for fid in list(rng.integers(sizes[2], sizes[3], 40)) + [sizes[2], sizes[3] - 1]:
        lv, op, a, b = sp.decode(int(fid))
        assert lv == 3
        if op <= 3:
            lo, hi = sorted((a, b))
            assert lo < sizes[1] <= hi < sizes[2]
        else:
            assert sizes[1] <= a < sizes[2] and b == -1
