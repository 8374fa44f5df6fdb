"""The learned form's pipeline through the C ABI: training set, training, evaluation.

Training data are the method's own exhaustive results: for each training problem, one SIS
step of the GPU path (k features), their FP64 Gram on the GPU, and for every 3-prefix of
the k features the lowest RSS/SST among the 5-subsets extending it (exhaustive, on the
GPU).  The network learns log10 of that value from the prefix's inputs.  Evaluation runs
the full method to D = 5 and compares the learned search (a fraction of the subsets)
with the exhaustive one, which stays the judge.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from .sisso import MLP, PREC_FP32, Sisso, prefix_training


def problem_gram(P, k: int):
    """(G, b, syy, N, ids) of one SIS step of k features against y."""
    with Sisso(P.X, P.y, P.op_set, P.rung, k, 1, precision=PREC_FP32, grammar=P.grammar) as c:
        ids = c.sis_step(P.y, [], k)
        G, b, syy = c.subspace_gram(ids)
    return G, b, syy, P.X.shape[0], ids


def training_set(n_problems: int, k: int = 60, per_problem: int = 1024, top: int = 128, seed: int = 0):
    """Inputs (M x 20, float32) and targets (M, float32): per problem the `top` best
    prefixes and `per_problem` random others (prefixes with extensions only); the target is
    log10 of the prefix's best completion's RSS/SST minus that of its greedy completion."""
    rng = np.random.default_rng(seed)
    Xs, ts = [], []
    for p in range(n_problems):
        P = inputs.workload4(p, held_out=False)
        G, b, syy, N, ids = problem_gram(P, k)
        if len(ids) < 5:
            continue
        X, lab, tgt = prefix_training(G, b, syy, N)
        ok = np.flatnonzero(np.isfinite(lab))
        if ok.size == 0:
            continue
        best = ok[np.argsort(lab[ok])[:top]]
        rest = rng.choice(ok, size=min(per_problem, ok.size), replace=False)
        sel = np.unique(np.concatenate([best, rest]))
        Xs.append(X[sel])
        ts.append(tgt[sel])
    return np.concatenate(Xs), np.concatenate(ts)


def train(X, t, seed: int = 0, epochs: int = 8, batch: int = 2048, lr: float = 1e-3) -> tuple[MLP, float]:
    """Train on standardised targets, then fold the scale into the output layer (w3, b3), so
    the network returns corrections in log10 units; the loss returned is relative to the
    targets' variance (1.0: no better than their mean)."""
    net = MLP(seed)
    M = (X.shape[0] // batch) * batch
    mu, sd = float(t[:M].mean()), float(t[:M].std()) or 1.0
    loss = net.train(X[:M], (t[:M] - mu) / sd, epochs=epochs, batch=batch, lr=lr, seed=seed)
    p = net.params()
    n_w3 = 256
    p[-1 - n_w3:-1] *= sd
    p[-1] = p[-1] * sd + mu
    net.set_params(p)
    return net, loss


def evaluate(net: MLP, problems, frac: float = 0.01, k: int = 60):
    """Per held-out problem: the exhaustive and the learned D = 5 search on the subspace the
    method builds (5 SIS steps of k), and the fit's time to the D = 5 descriptor with and
    without the network."""
    out = []
    for P in problems:
        rec = {"name": P.name}
        with Sisso(P.X, P.y, P.op_set, P.rung, k, 5, precision=PREC_FP32, grammar=P.grammar) as c:
            t0 = time.perf_counter()
            plain = c.fit()
            rec["fit_plain_s"] = time.perf_counter() - t0
            rec["fit_plain_ms_device"] = c.stats()["ms_fit"]
            S = sum((c.sis(t) for t in range(1, len(plain) + 1)), [])
            if len(plain) < 5:
                rec["skipped"] = "fit stopped before D = 5"
                out.append(rec)
                continue
            G, b, syy = c.subspace_gram(S)
            t0 = time.perf_counter()
            pos_ex, rss_ex, ex_ex = c.l0_search(G, b, syy, 5, S, PREC_FP32)
            rec["exhaustive_s"] = time.perf_counter() - t0
            t0 = time.perf_counter()
            pos_l, rss_l, ex_l, npre = c.l0_learned(G, b, syy, S, net, frac)
            rec["learned_s"] = time.perf_counter() - t0
            rec.update(n=len(S), examined_exhaustive=ex_ex, examined_learned=ex_l, prefixes=npre,
                       recall=sorted(pos_l) == sorted(pos_ex), rss_exhaustive=rss_ex, rss_learned=rss_l)
            c.set_proposal(net, frac, certify=False)
            t0 = time.perf_counter()
            learned = c.fit()
            rec["fit_learned_s"] = time.perf_counter() - t0
            rec["fit_learned_ms_device"] = c.stats()["ms_fit"]
            rec["fit_learned_launches"] = c.stats()["launches"]
            c.set_proposal(net, frac, certify=True)
            certified = c.fit()
            rec["fit_certified_ms_device"] = c.stats()["ms_fit"]
            rec["certified_prefixes"] = c.stats()["certified_prefixes"]
            rec["certified_ids"] = certified[4].ids
            c.set_proposal(None)
            rec["plain_ids"], rec["learned_ids"] = plain[4].ids, learned[4].ids
            rec["same_descriptor"] = learned[4].ids == plain[4].ids
            rec["rmse_rel_diff"] = abs(learned[4].rmse - plain[4].rmse) / plain[4].rmse
        out.append(rec)
    return out
