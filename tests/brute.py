"""Brute-force helpers for the oracle pins (tiny inputs only).

Written independently of ``oracle/``: the feature space is built as explicit expression
trees straight from the pair rule of §2.1 (Eq. 2 plus the "regenerated pairs are not
new" remark), values come from numpy, scores from ``numpy.corrcoef`` and least squares
from ``numpy.linalg.lstsq``.
"""
from __future__ import annotations

import itertools

import numpy as np

BINARY = ["+", "-", "*", "/"]
UNARY = ["exp", "log", "sqrt", "^2", "^-1", "sin", "^3", "exp-"]
TABLE = BINARY + UNARY


def space(d: int, ops: list[str], rung: int, new_x_prev: bool = False):
    """Features as nested tuples, in canonical order (level, operator, operands)."""
    feats = [("x", i) for i in range(d)]
    sizes = [d]
    prev_prev = 0            # |phi_{l-2}|
    for level in range(1, rung + 1):
        P = len(feats)
        Q = prev_prev
        new = []
        for op in TABLE:
            if op not in ops:
                continue
            if op in BINARY:
                for i in range(P):
                    for j in range(P):
                        if i == j:
                            continue
                        if op != "/" and not i < j:
                            continue
                        if new_x_prev and level >= 3:
                            if (i < Q) == (j < Q):
                                continue
                        elif i < Q and j < Q:
                            continue
                        new.append((op, feats[i], feats[j]))
            else:
                for z in range(Q, P):
                    new.append((op, feats[z]))
        feats = feats + new
        prev_prev = P
        sizes.append(len(feats))
    return feats, sizes


def evaluate(f, X: np.ndarray) -> np.ndarray:
    if f[0] == "x":
        return X[:, f[1]].astype(np.float64)
    with np.errstate(all="ignore"):
        a = evaluate(f[1], X)
        op = f[0]
        if op in BINARY:
            b = evaluate(f[2], X)
            return {"+": a + b, "-": a - b, "*": a * b, "/": a / b}[op]
        return {"exp": np.exp(a), "log": np.log(a), "sqrt": np.sqrt(a), "^2": a * a,
                "^-1": 1.0 / a, "sin": np.sin(a), "^3": a * a * a, "exp-": np.exp(-a)}[op]


def to_str(f) -> str:
    if f[0] == "x":
        return f"x{f[1] + 1}"
    op = f[0]
    if op in BINARY:
        return f"({to_str(f[1])}{op}{to_str(f[2])})"
    a = to_str(f[1])
    return {"exp": f"exp({a})", "log": f"log({a})", "sqrt": f"sqrt({a})", "^2": f"({a})^2",
            "^-1": f"({a})^-1", "sin": f"sin({a})", "^3": f"({a})^3", "exp-": f"exp(-{a})"}[op]


def valid(v: np.ndarray, f=None, X=None) -> bool:
    """Validity; with the feature tree f and X given, also the identically-zero rule
    (root + or - whose operands cancel to rounding noise) and, recursively, the validity
    of every operand."""
    if not np.all(np.isfinite(v)) or np.max(np.abs(v)) > 1e12:
        return False
    if f is not None and f[0] in ("+", "-"):
        mag = np.abs(evaluate(f[1], X)) + np.abs(evaluate(f[2], X))
        if np.max(np.abs(v)) <= 1e-9 * np.max(mag):
            return False
    if not float(np.std(v)) > 1e-6 * float(np.max(np.abs(v))):
        return False
    if f is not None and f[0] != "x":
        return all(valid(evaluate(ch, X), ch, X) for ch in f[1:])
    return True


def abs_corr(v: np.ndarray, t: np.ndarray) -> float:
    return float(abs(np.corrcoef(v, t)[0, 1]))


def standardise(v: np.ndarray) -> np.ndarray:
    return (v - v.mean()) / v.std()


def sis(values: list[np.ndarray], target: np.ndarray, S_prev: list[int], k: int,
        ok: list[bool] | None = None, thr: float = 0.0) -> list[int]:
    """SIS step (§2.2 Eqs. 5-6) by brute force, with the tie-tolerant walk and the
    duplicate rule (standardised vectors equal up to sign within 1e-8).  ok[i]: validity
    of feature i (default: the value rules only).  thr > 0: the threshold variant (§2.2,
    last paragraph), the walk ends once the best remaining |corr| is at or below thr."""
    if ok is None:
        ok = [valid(v) for v in values]
    cand = [(abs_corr(v, target), i) for i, v in enumerate(values)
            if ok[i] and i not in S_prev]
    refs = [standardise(values[i]) for i in S_prev if ok[i]]
    remaining = sorted(cand, key=lambda c: (-c[0], c[1]))
    acc = []
    while remaining and len(acc) < k:
        m = remaining[0][0]
        if thr > 0 and m <= thr:
            break
        window = [c for c in remaining if c[0] >= m - 1e-9]
        pick = min(window, key=lambda c: c[1])
        remaining.remove(pick)
        z = standardise(values[pick[1]])
        if any(np.max(np.abs(z - r)) <= 1e-8 or np.max(np.abs(z + r)) <= 1e-8 for r in refs):
            continue
        refs.append(z)
        acc.append(pick[1])
    return acc


def rss_with_intercept(cols: np.ndarray, y: np.ndarray) -> float:
    A = np.column_stack([np.ones(len(y)), cols])
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    r = y - A @ c
    return float(r @ r)


def best_subset(cols: np.ndarray, y: np.ndarray, D: int, gid: list[int]):
    """Exhaustive l0 by lstsq over every D-subset of the columns; tie rule on RSS within
    1e-12 * SST goes to the smallest ascending global-id tuple."""
    sst = float(((y - y.mean()) ** 2).sum())
    res = []
    for sub in itertools.combinations(range(cols.shape[1]), D):
        res.append((rss_with_intercept(cols[:, sub], y), tuple(sorted(gid[s] for s in sub)), sub))
    m = min(r[0] for r in res)
    tied = [r for r in res if r[0] <= m + 1e-12 * sst]
    return min(tied, key=lambda r: r[1]), len(res)


def sisso(X: np.ndarray, y: np.ndarray, d: int, ops: list[str], rung: int, k: int, T: int,
          new_x_prev: bool = False, thr: float = 0.0, stop_rmse: float = 0.0, W=None):
    """The whole iteration of §2.3 (Eq. 8) by brute force: SIS on y, then on the residual
    of the best t-term lstsq fit; l0 over all t-subsets of S_t.  thr: threshold SIS;
    stop_rmse: stop after a step whose RMSE is at or below it.  W: whitening (§2.4), every
    feature valid on the samples is mapped to W v (and must pass the value rules there),
    the target to W y, and the iteration runs on those."""
    feats, _ = space(d, ops, rung, new_x_prev)
    values = [evaluate(f, X) for f in feats]
    ok = [valid(v, f, X) for v, f in zip(values, feats)]
    if W is not None:
        values = [W @ v if o else v for v, o in zip(values, ok)]
        ok = [o and valid(v) for v, o in zip(values, ok)]
        y = W @ y
    S: list[int] = []
    out = []
    target = y.copy()
    for t in range(1, T + 1):
        S = S + sis(values, target, S, k, ok, thr)
        if len(S) < t:
            break
        cols = np.column_stack([values[i] for i in S])
        (rss, tup, sub), _ = best_subset(cols, y, t, S)
        A = np.column_stack([np.ones(len(y))] + [values[i] for i in tup])
        c, *_ = np.linalg.lstsq(A, y, rcond=None)
        target = y - A @ c
        rmse = float(np.sqrt(target @ target / len(y)))
        out.append((list(tup), c, rmse, list(S)))
        if rmse <= 1e-10 * y.std() or (stop_rmse > 0 and rmse <= stop_rmse):
            break
    return out


def units(f, labels):
    """Units of feature tree f as {label: exponent} (Fractions), or None when the tree
    breaks the dimensional rule: + and - on unequal units, exp, log, sin or exp- of a
    dimensioned operand.  labels[i]: unit label of primary i, -1 dimensionless."""
    from fractions import Fraction
    if f[0] == "x":
        lab = labels[f[1]]
        return {} if lab < 0 else {lab: Fraction(1)}
    a = units(f[1], labels)
    if a is None:
        return None
    op = f[0]
    if op in BINARY:
        b = units(f[2], labels)
        if b is None:
            return None
        if op in ("+", "-"):
            return a if a == b else None
        sign = 1 if op == "*" else -1
        out = dict(a)
        for k, v in b.items():
            out[k] = out.get(k, 0) + sign * v
        return {k: v for k, v in out.items() if v != 0}
    if op in ("exp", "log", "sin", "exp-"):
        return {} if not a else None
    scale = {"sqrt": Fraction(1, 2), "^2": 2, "^3": 3, "^-1": -1}[op]
    return {k: v * scale for k, v in a.items()}
