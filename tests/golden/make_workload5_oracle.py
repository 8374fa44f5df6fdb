"""Writes workload5_oracle.jsonl: the FP64 oracle's descriptors for the 512 seeded tasks of
the batched multi-task workload (N ~ U{20..2000}, d ~ U{4..12}, rung 2, nine operators,
k = 50, D <= 3).  Calls only ``oracle`` and the seeded input generators.

    python tests/golden/make_workload5_oracle.py [n_tasks]
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2410_01752_gb300 import inputs  # noqa: E402


def main(n_tasks: int = 512) -> None:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload5_oracle.jsonl")
    with open(out + ".tmp", "w") as f:
        for p in range(n_tasks):
            P = inputs.workload5_task(p)
            r = oracle.fit(P.X, P.y, oracle.Space(P.d, P.op_set, P.rung, P.grammar), P.sis_size, P.max_dim)
            rec = {"task": p, "N": int(P.X.shape[0]), "d": int(P.d),
                   "dims": [{"ids": [int(i) for i in D.ids], "coef": [float(c) for c in D.coef],
                             "rmse": float(D.rmse), "r2": float(D.r2)} for D in r.dims]}
            f.write(json.dumps(rec) + "\n")
            f.flush()
    os.replace(out + ".tmp", out)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 512)
