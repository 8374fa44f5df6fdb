"""Writes the FP64 oracle's full SISSO fits (§2.3 Eq. 8) of the seeded benchmark workloads
as golden files: per SIS step the accepted ids in acceptance order, per dimension the
descriptor's ids, coefficients (intercept first), RMSE, R^2, Gram-form RSS and the number
of subsets examined.  Calls only ``oracle`` and the seeded input generators.

    python tests/golden/make_fit_oracle.py CASE [CASE ...]

Cases (file ``<case>_oracle.json`` beside this script):
  workload2      N=1000, d=10, lognormal primaries, rung 3 (NEW_X_PREV), k=100, D<=4
  workload2_d6   the same recipe at d=6 (a smaller rung-3 space, same N, k and D)
  workload3      N=65536, d=12, six primaries correlated 0.999, rung 2, k=200, D<=3
  workload4      held-out learned-proposal problems 0..7: rung 2, k=60, D<=5
                 (the D = 5 step searches C(300, 5) subsets)
  ensemble       the 30 disjoint 100-sample subsets (partition seed 0) of the four-term
                 ensemble problem (§4.5): rung 2, k=20, D<=4
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2410_01752_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    "workload2": [("workload2", 0, {})],
    "workload2_d6": [("workload2", 0, {"d": 6})],
    "workload3": [("workload3", 0, {})],
    "workload4": [("workload4", p, {"held_out": True}) for p in range(8)],
    "ensemble": [("ensemble_problem", 0, {}, (30, 100, 0, m)) for m in range(30)],
}


def fit_record(gen: str, p: int, kw: dict, part=None) -> dict:
    """part = (n_models, size, seed, m): the fit of subset m of inputs.partition_rows."""
    P = getattr(inputs, gen)(p, **kw)
    X, y = P.X, P.y
    if part is not None:
        rows = inputs.partition_rows(P.N, part[0], part[1], part[2])[part[3]]
        X, y = X[rows], y[rows]
    t0 = time.time()
    r = oracle.fit(X, y, oracle.Space(P.d, P.op_set, P.rung, P.grammar), P.sis_size, P.max_dim)
    return {
        "generator": gen, "p": p, "kwargs": kw, "name": P.name, "partition": part,
        "N": int(X.shape[0]), "d": int(P.d), "op_set": int(P.op_set), "rung": int(P.rung),
        "grammar": int(P.grammar), "sis_size": int(P.sis_size), "max_dim": int(P.max_dim),
        "sis": [[int(i) for i in s] for s in r.sis],
        "dims": [{"ids": [int(i) for i in D.ids], "coef": [float(c) for c in D.coef],
                  "rmse": float(D.rmse), "r2": float(D.r2), "rss_gram": float(D.rss_gram),
                  "subsets": int(D.subsets)} for D in r.dims],
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": len(os.sched_getaffinity(0)),
    }


def main(names) -> None:
    for name in names:
        out = os.path.join(HERE, f"{name}_oracle.json")
        recs = []
        for case in CASES[name]:
            recs.append(fit_record(*case))
            print(name, case[1], case[3:] or "", recs[-1]["oracle_seconds"], "s", flush=True)
            with open(out + ".tmp", "w") as f:       # partial results survive an interruption
                json.dump(recs, f, indent=1)
        os.replace(out + ".tmp", out)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
