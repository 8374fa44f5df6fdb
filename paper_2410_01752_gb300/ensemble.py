"""Resampled fits through the batched form: ensembles and k-fold validation.

The paper recommends k-fold cross-validation for small data sets and bootstrap aggregation
(bagging) for robustness to noise (§2.4, closing paragraphs), and trains an ensemble of
models on disjoint partitions of one data set as independent GPU tasks (§4.5, the ensemble
timing table).  Here every resampled copy of the problem is one task of the batched form
(one persistent launch, ``sisso.Batch``): the fits run in the library's kernels; this module
takes the row sets (seeded, from ``inputs``, passed to the fits as inputs), gathers each
task's rows as its host input, and evaluates the fitted descriptors
(``Sisso.eval_features``, FP64 on the device) to combine predictions.

Readings (the paper fixes none of them): a bootstrap sample has N rows drawn uniformly with
replacement; the bagged prediction is the mean of the models' predictions at their last
dimension; the k folds are the contiguous slices of one seeded permutation of the rows, the
first N mod k folds one row longer; the cross-validated RMSE of dimension t pools every
held-out squared error of the folds' dimension-t models.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import sisso
from .inputs import bootstrap_rows, kfold_rows, partition_rows  # noqa: F401  (seeded row sets)


# ---- fits and predictions --------------------------------------------------------------
@dataclass
class Model:
    rows: np.ndarray                  # training rows
    status: int
    dims: list                        # [sisso.Descriptor for t = 1..n_dims]


def fit_rows(X, y, row_sets, op_set: int, rung: int, sis_size: int, max_dim: int,
             grammar: int = sisso.GRAMMAR_EQ2, stream=None) -> list[Model]:
    """Fit every row set as one task of one batched launch."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    probs = [(X[r], y[r]) for r in row_sets]
    with sisso.Batch(probs, op_set, rung, sis_size, max_dim, grammar=grammar, stream=stream) as b:
        b.run()
        res = b.results()
    return [Model(np.asarray(r), st, dims) for r, (st, dims) in zip(row_sets, res)]


def predict(X, y, models: list[Model], op_set: int, rung: int, grammar: int = sisso.GRAMMAR_EQ2,
            dim: int | None = None) -> np.ndarray:
    """Predictions (n_models x N) of each model's dimension-`dim` descriptor (default: its last)
    on every row of X; NaN rows for models without a descriptor."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.full((len(models), X.shape[0]), np.nan)
    want = []
    for m in models:
        t = (len(m.dims) if dim is None else dim) if m.status == 0 else 0
        want.append(m.dims[t - 1] if 1 <= t <= len(m.dims) else None)
    ids = sorted({i for d in want if d is not None for i in d.ids})
    if not ids:
        return out
    with sisso.Sisso(X, y, op_set, rung, 1, 1, grammar=grammar) as c:
        vals = c.eval_features(np.array(ids, dtype=np.int64))
    row = {i: v for i, v in zip(ids, vals)}
    for m, d in enumerate(want):
        if d is not None:
            out[m] = d.coef[0] + sum(cf * row[i] for cf, i in zip(d.coef[1:], d.ids))
    return out


@dataclass
class Bagged:
    models: list[Model]
    prediction: np.ndarray            # mean over models of their last-dimension predictions
    rmse: float                       # of the bagged prediction on every row
    descriptor_counts: dict           # (ids of the last dimension) -> models that chose it


def bagging(X, y, op_set: int, rung: int, sis_size: int, max_dim: int, n_models: int, seed: int,
            grammar: int = sisso.GRAMMAR_EQ2, stream=None) -> Bagged:
    """Bootstrap aggregation: n_models bootstrap fits in one launch, their mean prediction."""
    rows = bootstrap_rows(len(y), n_models, seed)
    models = fit_rows(X, y, rows, op_set, rung, sis_size, max_dim, grammar, stream)
    P = predict(X, y, models, op_set, rung, grammar)
    ok = ~np.isnan(P).any(axis=1)
    pred = P[ok].mean(axis=0) if ok.any() else np.full(len(y), np.nan)
    counts: dict = {}
    for m in models:
        if m.status == 0 and m.dims:
            key = tuple(m.dims[-1].ids)
            counts[key] = counts.get(key, 0) + 1
    return Bagged(models, pred, float(np.sqrt(np.mean((np.asarray(y) - pred) ** 2))), counts)


@dataclass
class CrossValidation:
    folds: list[tuple[np.ndarray, np.ndarray]]
    models: list[Model]
    rmse: list[float]                 # pooled held-out RMSE per dimension t = 1..max_dim
    fold_rmse: np.ndarray             # K x max_dim held-out RMSE (NaN where a fold has no model)


def kfold(X, y, op_set: int, rung: int, sis_size: int, max_dim: int, K: int, seed: int,
          grammar: int = sisso.GRAMMAR_EQ2, stream=None) -> CrossValidation:
    """k-fold cross-validation: the K training folds fitted in one launch, each dimension's
    model scored on its held-out rows."""
    y = np.asarray(y, dtype=np.float64)
    folds = kfold_rows(len(y), K, seed)
    models = fit_rows(X, y, [tr for tr, _ in folds], op_set, rung, sis_size, max_dim, grammar, stream)
    fold_rmse = np.full((K, max_dim), np.nan)
    sq = [[] for _ in range(max_dim)]
    for t in range(1, max_dim + 1):
        P = predict(X, y, models, op_set, rung, grammar, dim=t)
        for f, (_, te) in enumerate(folds):
            if not np.isnan(P[f]).any() and len(models[f].dims) >= t:
                e = y[te] - P[f][te]
                fold_rmse[f, t - 1] = float(np.sqrt(np.mean(e * e)))
                sq[t - 1].append(e * e)
    rmse = [float(np.sqrt(np.mean(np.concatenate(s)))) if s else float("nan") for s in sq]
    return CrossValidation(folds, models, rmse, fold_rmse)
