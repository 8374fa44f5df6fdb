"""Seeded synthetic inputs shaped like the paper's workloads (numpy only).

This module makes data and nothing else: it holds none of the method's arithmetic and is
shared by the tests, the benchmark and the smoke check.  Problem ``p`` of workload ``c``
draws from ``numpy.random.default_rng(1000 * c + p)`` (PCG64).

Workloads (x: primary features, N samples x d; y: target):
  1  N=50, d=5, x ~ U[1,5]; y = 3 x1 x2 / x3 + 0.5 + N(0, 0.01^2)            (rung 2, k=20, D<=3)
  2  N=1000, d=10, x ~ lognormal(0, 0.5); y = sum_m c_m f_m + 1% noise with
     f1 = x1 x2 / x3, f2 = (x4 + x5)^2 / x6, f3 = log(x7) x8 / (x9 + x10),
     c ~ U(-5, 5), noise sd = 0.01 std(clean)                                  (rung 3, k=100, D<=4)
  3  N=65536, d=12; x7..x12 ~ U[1,5]; x1..x6 = 3 + 0.5 (sqrt(.999) g + sqrt(.001) e_j)
     (pairwise correlation 0.999); y = c1 x1 x7^2 + c2 x2 / sqrt(x8) + c3 log(x3) x9
     + 1% noise                                                                 (rung 2, k=200, D<=3)
  4  learned proposal: problem p of the training set (seeds 4000 + p) or of the held-out
     evaluation set (seeds 40000 + p): N ~ U{500..2000}, d ~ U{8..12}, x ~ U[1,5],
     3-5 distinct planted rung-2 terms from the menu below, c ~ U(-5, 5), 1% noise
                                                                                (rung 2, k=60, D<=5)
  5  one of 512 tasks: N ~ U{20..2000}, d ~ U{4..12}, x ~ U[0.5, 5], 1-3 planted rung-2
     terms from a fixed menu, c ~ U(-5, 5), 0.5% noise                          (rung 2, k=50, D<=3)
  6  the ensemble timing workload (§4.5): N=3000, d=4, x ~ U[1,5], y = x1^4 + x2^3 + x3^2
     + x4 + 0.1% noise, cut into 30 subsets of 100 samples                       (rung 2, k=20, D<=4)
  7  whitening (§2.4): N=500, d=5, x ~ U[1,5]; y = 2 x1 x2 / x3 + sqrt(x5) + AR(1) noise
     (coefficient 0.6, innovations sd 0.05), with the whitening matrix of that covariance
     (the Prais-Winsten transform, lower bidiagonal)                           (rung 2, k=10, D<=3)
  The paper's own workloads are of the same kind: x in [1,5], small N, 3-4 term targets
  (§4.1, §4.5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# operator bits (order of the public operator table)
ADD, SUB, MUL, DIV, EXP, LOG, SQRT, SQ, INV, SIN, CUBE, EXPNEG = range(12)
OPS9 = sum(1 << o for o in (ADD, SUB, MUL, DIV, EXP, LOG, SQRT, SQ, INV))
GRAMMAR_EQ2, GRAMMAR_NEW_X_PREV = 0, 1


@dataclass
class Problem:
    X: np.ndarray          # N x d, float64, row-major
    y: np.ndarray          # N, float64
    op_set: int
    rung: int
    sis_size: int
    max_dim: int
    grammar: int
    name: str

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def _rng(config: int, p: int) -> np.random.Generator:
    return np.random.default_rng(1000 * config + p)


def workload1(p: int = 0, N: int = 50) -> Problem:
    r = _rng(1, p)
    X = r.uniform(1.0, 5.0, size=(N, 5))
    y = 3.0 * X[:, 0] * X[:, 1] / X[:, 2] + 0.5 + r.normal(0.0, 0.01, size=N)
    return Problem(X, y, OPS9, 2, 20, 3, GRAMMAR_EQ2, "plain-fp64 N=50 d=5 rung2 k=20 D<=3")


def workload2(p: int = 0, N: int = 1000, d: int = 10, sis_size: int = 100, max_dim: int = 4,
              rung: int = 3) -> Problem:
    r = _rng(2, p)
    X = r.lognormal(0.0, 0.5, size=(N, d))
    x = [X[:, j] for j in range(d)]
    c = r.uniform(-5.0, 5.0, size=3)
    if d >= 10:
        f = [x[0] * x[1] / x[2], (x[3] + x[4]) ** 2 / x[5], np.log(x[6]) * x[7] / (x[8] + x[9])]
    else:                  # reduced-size variants keep the same shapes of terms
        f = [x[0] * x[1] / x[2 % d], (x[3 % d] + x[1]) ** 2 / x[0], np.log(x[2 % d]) * x[1]]
    clean = sum(ci * fi for ci, fi in zip(c, f))
    y = clean + r.normal(0.0, 0.01 * clean.std(), size=N)
    return Problem(X, y, OPS9, rung, sis_size, max_dim, GRAMMAR_NEW_X_PREV,
                   f"plain-fp32 N={N} d={d} rung{rung} k={sis_size} D<={max_dim}")


def workload3(p: int = 0, N: int = 65536, sis_size: int = 200, max_dim: int = 3) -> Problem:
    r = _rng(3, p)
    X = np.empty((N, 12))
    g = r.normal(size=N)
    for j in range(6):
        X[:, j] = 3.0 + 0.5 * (np.sqrt(0.999) * g + np.sqrt(0.001) * r.normal(size=N))
    X[:, 6:] = r.uniform(1.0, 5.0, size=(N, 6))
    c = r.uniform(-5.0, 5.0, size=3)
    clean = (c[0] * X[:, 0] * X[:, 6] ** 2 + c[1] * X[:, 1] / np.sqrt(X[:, 7])
             + c[2] * np.log(X[:, 2]) * X[:, 8])
    y = clean + r.normal(0.0, 0.01 * clean.std(), size=N)
    return Problem(X, y, OPS9, 2, sis_size, max_dim, GRAMMAR_EQ2,
                   f"mixed N={N} d=12 collinear rung2 k={sis_size} D<={max_dim}")


def ensemble_problem(p: int = 0, N: int = 3000, sis_size: int = 20, max_dim: int = 4) -> Problem:
    """The ensemble timing workload (§4.5): the first four-term model x1^4 + x2^3 + x3^2 + x4,
    x ~ U[1, 5], 3000 samples to be cut into 30 subsets of 100, k = 20 (noise 0.1% of the
    clean signal's std, so that no two descriptors fit exactly)."""
    r = _rng(6, p)
    X = r.uniform(1.0, 5.0, size=(N, 4))
    clean = X[:, 0] ** 4 + X[:, 1] ** 3 + X[:, 2] ** 2 + X[:, 3]
    y = clean + r.normal(0.0, 1e-3 * clean.std(), size=N)
    return Problem(X, y, OPS9, 2, sis_size, max_dim, GRAMMAR_EQ2,
                   f"ensemble four-term N={N} d=4 rung2 k={sis_size} D<={max_dim}")


@dataclass
class WhitenedProblem(Problem):
    W: np.ndarray = None   # N x N whitening matrix of the noise covariance (W Sigma W^T = I)


def ar1_whitener(N: int, rho: float, sd: float) -> np.ndarray:
    """The whitening matrix of AR(1) noise e_t = rho e_{t-1} + u_t, u ~ N(0, sd^2), stationary
    start (the Prais-Winsten transform): row 0 = sqrt(1 - rho^2) e_0 / sd, row t = (e_t - rho
    e_{t-1}) / sd, so that W e has independent unit-variance entries."""
    W = np.zeros((N, N))
    W[0, 0] = np.sqrt(1.0 - rho * rho) / sd
    i = np.arange(1, N)
    W[i, i] = 1.0 / sd
    W[i, i - 1] = -rho / sd
    return W


def whitened_problem(p: int = 0, N: int = 500, sis_size: int = 10, max_dim: int = 3,
                     rho: float = 0.6, sd: float = 0.05) -> WhitenedProblem:
    """Workload 7: a planted rung-2 target with AR(1) noise and its whitening matrix."""
    r = _rng(7, p)
    X = r.uniform(1.0, 5.0, size=(N, 5))
    e = np.empty(N)
    e[0] = r.normal(0.0, sd / np.sqrt(1.0 - rho * rho))
    u = r.normal(0.0, sd, size=N)
    for t in range(1, N):
        e[t] = rho * e[t - 1] + u[t]
    y = 2.0 * X[:, 0] * X[:, 1] / X[:, 2] + np.sqrt(X[:, 4]) + e
    return WhitenedProblem(X, y, OPS9, 2, sis_size, max_dim, GRAMMAR_EQ2,
                           f"whitened AR(1) N={N} d=5 rung2 k={sis_size} D<={max_dim}", ar1_whitener(N, rho, sd))


_MENU = [
    lambda x: x[0] * x[1] / x[2],
    lambda x: np.sqrt(x[0]) * x[3],
    lambda x: (x[1] + x[2]) ** 2,
    lambda x: np.log(x[3]) / x[0],
    lambda x: x[2] * x[2] / x[1],
    lambda x: np.exp(x[0] / x[3]),
    lambda x: (x[0] - x[1]) * x[2],
    lambda x: 1.0 / (x[1] * x[3]),
]


def workload5_task(p: int) -> Problem:
    r = _rng(5, p)
    N = int(r.integers(20, 2001))
    d = int(r.integers(4, 13))
    X = r.uniform(0.5, 5.0, size=(N, d))
    perm = r.permutation(d)
    x = [X[:, perm[j]] for j in range(4)]
    terms = r.choice(len(_MENU), size=int(r.integers(1, 4)), replace=False)
    c = r.uniform(-5.0, 5.0, size=len(terms))
    clean = sum(ci * _MENU[t](x) for ci, t in zip(c, terms))
    y = clean + r.normal(0.0, 0.005 * max(clean.std(), 1e-12), size=N)
    return Problem(X, y, OPS9, 2, 50, 3, GRAMMAR_EQ2, f"task{p} N={N} d={d}")


def workload4(p: int, held_out: bool = True, sis_size: int = 60, max_dim: int = 5) -> Problem:
    r = np.random.default_rng((40000 if held_out else 4000) + p)
    N = int(r.integers(500, 2001))
    d = int(r.integers(8, 13))
    X = r.uniform(1.0, 5.0, size=(N, d))
    perm = r.permutation(d)
    x = [X[:, perm[j]] for j in range(4)]
    terms = r.choice(len(_MENU), size=int(r.integers(3, 6)), replace=False)
    c = r.uniform(-5.0, 5.0, size=len(terms))
    clean = sum(ci * _MENU[t](x) for ci, t in zip(c, terms))
    y = clean + r.normal(0.0, 0.01 * max(clean.std(), 1e-12), size=N)
    return Problem(X, y, OPS9, 2, sis_size, max_dim, GRAMMAR_EQ2,
                   f"learned-{'eval' if held_out else 'train'}{p} N={N} d={d} rung2 k={sis_size} D<={max_dim}")


# row sets of resampled fits (ensembles, bagging, k-fold; §2.4, §4.5): data selection only
def partition_rows(N: int, n_models: int, size: int, seed: int) -> list[np.ndarray]:
    """Disjoint subsets of `size` rows each (one seeded permutation, cut in order)."""
    if n_models * size > N:
        raise ValueError("partition needs n_models * size <= N")
    perm = np.random.default_rng(seed).permutation(N)
    return [np.sort(perm[m * size:(m + 1) * size]) for m in range(n_models)]


def bootstrap_rows(N: int, n_models: int, seed: int, size: int | None = None) -> list[np.ndarray]:
    """Bootstrap samples: `size` (default N) rows drawn uniformly with replacement."""
    r = np.random.default_rng(seed)
    n = N if size is None else size
    return [np.sort(r.integers(0, N, n)) for _ in range(n_models)]


def kfold_rows(N: int, K: int, seed: int) -> list[tuple[np.ndarray, np.ndarray]]:
    """(training rows, held-out rows) of each of K folds."""
    if not 2 <= K <= N:
        raise ValueError("k-fold needs 2 <= K <= N")
    perm = np.random.default_rng(seed).permutation(N)
    sizes = [N // K + (1 if f < N % K else 0) for f in range(K)]
    out, at = [], 0
    for f in range(K):
        test = np.sort(perm[at:at + sizes[f]])
        at += sizes[f]
        out.append((np.setdiff1d(np.arange(N), test), test))
    return out


def workload(config: int, p: int = 0, **kw) -> Problem:
    return {1: workload1, 2: workload2, 3: workload3, 4: workload4, 5: workload5_task,
            6: ensemble_problem}[config](p, **kw)
