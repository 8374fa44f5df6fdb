#!/usr/bin/env python3
"""Benchmark of the SISSO hot path on GB300.

One step = one whole SISSO fit (§2.3 Eq. 8): for t = 1..4, SIS screening of every
candidate of the rung-3 feature space (2.91e8 ids: 1000 samples x 10 lognormal primaries,
one rung-3 operand from phi_1) plus the exhaustive l0 over all t-subsets of S_t
(k = 100 per step, C(400, 4) = 1.05e9 subsets at t = 4).  Inputs are resident in HBM
before the timed region; between timed steps L2 is flushed by writing 256 MB.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun (N > 1) every rank fits its own seeded problem (independent replicas,
weak scaling); the step time is the maximum over ranks.  ``--impl reference`` times the
FP64 CPU oracle (the reference of this method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "features scored/s, ℓ0 subsets fit/s; time-to-descriptor vs plain at equal RMSE"
UNIT = "features/s"
FP32_FLOP_PER_CAND_SAMPLE = 6          # op, add, 2 FMA (sum, sum of squares, cross)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU work for the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="default line: skip the bounded runs of the mixed, batched and learned forms")
    ap.add_argument("--workload", type=int, default=2, choices=[2, 3, 4, 5, 7],
                    help="2: rung-3 screening + l0 (default); 3: mixed precision vs plain, 65 536 samples; "
                         "7: whitened fit (AR(1) noise, 500 samples)")
    ap.add_argument("--tasks", type=int, default=512, help="batched workload: number of tasks")
    ap.add_argument("--train-problems", type=int, default=2000, help="learned workload: training problems")
    ap.add_argument("--eval-problems", type=int, default=100, help="learned workload: held-out problems")
    ap.add_argument("--frac", type=float, default=0.01, help="learned workload: fraction of subsets solved")
    ap.add_argument("--tune-cache", default=None, help="batched workload: autotuner cache file")
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: default launch shape")
    ap.add_argument("--d", type=int, default=10, help="primary features (smaller cases for profiling)")
    ap.add_argument("--N", type=int, default=1000, help="samples (smaller cases for profiling)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi samples every 200 ms while running (clocks and throttle reasons)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_baseline_sample(P, seconds: float, seed: int = 0, threads: int = 0):
    """The FP64 oracle scoring a random sample of the workload's candidate ids on all host
    cores (or `threads`); returns (features/s, ids scored, wall seconds, threads)."""
    import numpy as np
    import oracle
    sp = oracle.Space(P.d, P.op_set, P.rung, P.grammar)
    n = sp.n_features
    rng = np.random.default_rng(seed)
    th = threads if threads > 0 else cores()
    probe = rng.integers(0, n, 2000)
    t0 = time.perf_counter()
    sp.scores(P.X, P.y, probe, nthreads=th)
    dt = max(time.perf_counter() - t0, 1e-3)
    m = int(max(2000, min(5e7, 2000 * seconds / dt)))
    ids = rng.integers(0, n, m)
    t0 = time.perf_counter()
    sp.scores(P.X, P.y, ids, nthreads=th)
    dt = time.perf_counter() - t0
    return m / dt, m, dt, th


def captured_traffic():
    """DRAM bytes per launch of the pair kernel from the committed ncu summary, or None
    when the kernel's source has changed since that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_score_pairs_rung3_N1000_d10_traffic.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in txt.splitlines() if l.startswith(("traffic_bytes", "source_sha256")))
    h = hashlib.sha256()
    for f in ("sis.cu", "sis_device.cuh"):        # the kernel, its device code and its tile list
        with open(os.path.join(ROOT, "paper_2410_01752_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    sha = next((v.strip() for k, v in vals.items() if k.startswith("source_sha256")), "")
    if sha != h.hexdigest():
        return None
    return int(vals["traffic_bytes_per_launch"].strip())


def captured_batch_traffic(tune: dict):
    """DRAM bytes per launch of the batched kernel from the committed ncu summary, or None
    when its source or the launch shape differs from that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_batch_workload5_512tasks_traffic.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in txt.splitlines()
                if l.startswith(("traffic_bytes", "source_sha256", "tune")))
    h = hashlib.sha256()
    for f in ("batch.cu", "sis_device.cuh", "l0_device.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2410_01752_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    sha = next((v.strip() for k, v in vals.items() if k.startswith("source_sha256")), "")
    shape = [tune[k] for k in ("score_units", "enum_items", "gram_rows", "ctas_per_sm", "window")]
    if sha != h.hexdigest() or [int(x) for x in vals.get("tune", "").split()] != shape:
        return None
    return int(vals["traffic_bytes_per_launch"].strip())


def job_totals(total_ms, counts, dist, device):
    """Whole-job figures of a replicated run: the slowest rank's time (the job ends when it
    does) and every rank's units summed.  dist None: a single process."""
    if dist is None:
        return float(total_ms), [float(v) for v in counts]
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(v) for v in counts], device=device, dtype=torch.float64)
    dist.all_reduce(c)
    return float(t.item()), [float(v) for v in c.tolist()]


def top_binary_candidates(sizes, n_unary_ops):
    """Candidates of the top level's binary sections (the pair kernel's work)."""
    L = len(sizes) - 1
    P, Q = sizes[L - 1], (sizes[L - 2] if L >= 2 else 0)
    return sizes[L] - P - (P - Q) * n_unary_ops


GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden_fit(name):
    """The oracle's stored fits of a workload (tests/golden/<name>_oracle.json), or None."""
    try:
        with open(os.path.join(GOLDEN, f"{name}_oracle.json")) as f:
            return json.load(f)
    except OSError:
        return None


def compare_fit(sis_steps, desc, rec, rtol):
    """Parity of one fit against the oracle's stored fit: SIS selections and descriptors
    bit-exact, coefficients and RMSE within rtol relative."""
    out = {"sis_steps_equal": [list(a) for a in sis_steps] == rec["sis"],
           "descriptors_equal": [d.ids for d in desc] == [r["ids"] for r in rec["dims"]],
           "coef_max_rel_err": None, "rmse_max_rel_err": None}
    if out["descriptors_equal"]:
        ce = [abs(a - b) / max(abs(b), 1e-300) for d, r in zip(desc, rec["dims"]) for a, b in zip(d.coef, r["coef"])]
        re = [abs(d.rmse - r["rmse"]) / r["rmse"] for d, r in zip(desc, rec["dims"]) if r["rmse"] > 0]
        out["coef_max_rel_err"], out["rmse_max_rel_err"] = max(ce), max(re) if re else 0.0
    out["ok"] = bool(out["sis_steps_equal"] and out["descriptors_equal"] and out["coef_max_rel_err"] <= rtol
                     and out["rmse_max_rel_err"] <= rtol)
    out["tolerance_rel"] = rtol
    return out


L0_FLOP_PER_SUBSET = {1: 3, 2: 11, 3: 26, 4: 50, 5: 85}   # full Cholesky solve + RSS per D-subset (FMA = 2)
L0_FP32_OPS_PER_SUBSET = {3: 8, 4: 9, 5: 10}              # tiled enumeration: FP32 arithmetic per subset (filter included)


_ALU_PEAK = {}


def alu_peak(sms, mhz):
    """The FP32 pipe's peak for the ALU-bound kernels' roofline: derived from the unit counts
    and the clock (SMs x 128 FP32 lanes x 2 flop x max SM clock), with the FMA rates measured
    once before any timed region (sisso_measure_alu_peak: FP32, paired FP32, FP64; every SM
    busy, CUDA events) reported beside it."""
    if not _ALU_PEAK:
        from paper_2410_01752_gb300 import sisso
        derived = sms * 128 * 2 * mhz * 1e6 / 1e12
        try:
            f32 = sisso.measure_alu_peak(sisso.ALU_FP32)
            f32x2 = sisso.measure_alu_peak(sisso.ALU_FP32X2)
            f64 = sisso.measure_alu_peak(sisso.ALU_FP64)
            _ALU_PEAK.update(peak=derived, fp32=f32, fp32x2=f32x2, fp64=f64, derived=derived,
                             source=f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz (measured max "
                                    f"SM clock) = {derived:.1f}; measured FMA rates (sisso_measure_alu_peak): FP32 "
                                    f"{f32:.1f}, paired FP32 {f32x2:.1f}, FP64 {f64:.2f} TFLOP/s")
        except Exception as e:      # noqa: BLE001
            _ALU_PEAK.update(peak=derived, derived=derived,
                             source=f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz ({e})")
    return _ALU_PEAK


def l0_roofline(s, D, peak, sms, mhz, reps=3):
    """The tiled l0 enumeration alone, one launch over every D-subset of the fit's final
    subspace (the fit's own last step), timed with CUDA events inside the library."""
    import math
    import numpy as np
    S = sum((s.sis(t) for t in range(1, D + 1)), [])
    G, b, syy = s.subspace_gram(S)
    ms = []
    for _ in range(reps):
        st0 = s.stats()
        s.l0_search(G, b, syy, D, np.array(S))
        st1 = s.stats()
        ms.append(st1["ms_l0_enum"] - st0["ms_l0_enum"])
        cand = st1["l0_candidates"] - st0["l0_candidates"]
    t = sorted(ms)[len(ms) // 2] / 1e3
    n_sub = math.comb(len(S), D)
    achieved = L0_FLOP_PER_SUBSET[D] * n_sub / t / 1e12
    return {"bound": "alu", "kernel": f"k_l0_tile<{D - 2}>", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "launch_ms": t * 1e3, "subsets": n_sub,
            "subsets_per_s": n_sub / t, "candidates_exact_test": int(cand),
            "algorithmic_unit": f"{L0_FLOP_PER_SUBSET[D]} flop per {D}-subset (full Cholesky solve and RSS, FMA = 2) "
                                f"x C({len(S)},{D}) subsets per launch",
            "fp32_issue_frac": L0_FP32_OPS_PER_SUBSET.get(D, 0) * n_sub / t / (sms * 128 * mhz * 1e6),
            "fp32_issue_note": f"{L0_FP32_OPS_PER_SUBSET.get(D, 0)} FP32 arithmetic instructions per subset in the "
                               "prefix-reduced form, against SMs x 128 lanes x clock",
            "peak_source": alu_peak(sms, mhz)["source"]}


def sisso_sizes(P):
    from paper_2410_01752_gb300 import sisso
    return sisso.space_sizes(P.d, P.op_set, P.rung, P.grammar)


def form_mixed(args):
    """Mixed-precision forms vs the plain FP32 form at full size (65 536 samples, six
    primaries correlated 0.999, rung 2, k = 200, D <= 3): time to the final descriptor and
    parity of every form with the oracle's stored fit."""
    import torch
    from paper_2410_01752_gb300 import PREC_FP32, PREC_MIXED_BF16, PREC_MIXED_FP16, Sisso, inputs
    P = inputs.workload3(0)
    rec = (golden_fit("workload3") or [None])[0]
    Xd, yd = torch.from_numpy(P.X).cuda(), torch.from_numpy(P.y).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {}
    for name, prec, tol, gram in (("plain_fp32", PREC_FP32, 1e-6, 0), ("fp32_tf32x3_gram", PREC_FP32, 1e-6, 2),
                                  ("mixed_bf16", PREC_MIXED_BF16, 1e-4, 0), ("mixed_fp16", PREC_MIXED_FP16, 1e-4, 0)):
        with Sisso(Xd, yd, P.op_set, P.rung, P.sis_size, P.max_dim, precision=prec, grammar=P.grammar,
                   stream=stream, gram=gram) as s:
            s.fit()
            ms = []
            for _ in range(2):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                d = s.fit()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            st = s.stats()
            out[name] = {"time_to_descriptor_ms": sum(ms) / len(ms), "descriptor": d[-1].ids, "rmse": d[-1].rmse,
                         "gpu_launches": st["launches"],
                         "phase_ms": {k: st[k] for k in ("ms_screen", "ms_screen_pair", "ms_select", "ms_rescore",
                                                          "ms_walk", "ms_gram", "ms_l0", "ms_refit")},
                         "screen_tensor_cores": bool(st["screen_tc"]), "tc_keys_raised": st["tc_keys_raised"],
                         "survivors_rescored": st["survivors_rescored"],
                         "parity": compare_fit([s.sis(t) for t in range(1, len(d) + 1)], d, rec, tol) if rec else None}
            if st["screen_tc"]:
                # split 16-bit products of the screening: one target-independent product
                # (2 Pp x 4 Pp) per fit and one (Pp x 2 Pp) per step, K = padded samples x parts
                Pp = -(-int(sisso_sizes(P)[1]) // 128) * 128
                Kp = -(-P.N // 64) * 64
                parts = 6 if prec == PREC_MIXED_BF16 else 3
                flop = 2.0 * (8 * Pp * Pp + len(d) * 2 * Pp * Pp) * Kp * parts
                pk = peaks()
                out[name]["screen_tc_products"] = {
                    "flop_per_fit": flop, "tflops_over_pair_stage": flop / (st["ms_screen_pair"] / 1e3) / 1e12,
                    "note": "over the whole tensor-core pair stage (row preparation, products, chunk sums, keys)",
                    "bf16_peak_measured": pk.get("bf16_tflops")}
    for k in ("fp32_tf32x3_gram", "mixed_bf16", "mixed_fp16"):
        out[k]["speedup_vs_plain"] = out["plain_fp32"]["time_to_descriptor_ms"] / out[k]["time_to_descriptor_ms"]
        out[k]["rmse_rel_diff_vs_plain"] = abs(out[k]["rmse"] - out["plain_fp32"]["rmse"]) / out["plain_fp32"]["rmse"]
    cpu = None
    if not args.no_cpu_baseline:
        r, m, dt, th = cpu_baseline_sample(P, 5.0, seed=3)
        cpu = {"value": r, "unit": "features/s", "cores": th, "kind": "oracle",
               "sample": f"{m} random candidate ids scored in FP64 over all {P.N} samples ({dt:.1f} s)"}
    return {"workload": P.name, "forms": out, "cpu_baseline": cpu,
            "metric": "time-to-descriptor vs plain at equal RMSE", "unit": "ms",
            "parity_ok": all(v["parity"] and v["parity"]["ok"] for v in out.values())}


def form_ensemble(args):
    """The paper's ensemble timing workload (§4.5): 30 models, each fitted on a disjoint
    100-sample subset of the four-term problem (k = 20, D <= 4), as the 30 tasks of one
    batched launch; every model against the oracle's stored fit of its subset."""
    import numpy as np
    import torch
    from paper_2410_01752_gb300 import ensemble, inputs, sisso
    P = inputs.ensemble_problem(0)
    rows = inputs.partition_rows(P.N, 30, 100, 0)
    probs = [(P.X[r], P.y[r]) for r in rows]
    stream = torch.cuda.current_stream()
    with sisso.Batch(probs, P.op_set, P.rung, P.sis_size, P.max_dim, stream=stream) as b:
        b.run(copies=False)
        ms = []
        for _ in range(5):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(copies=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res = b.results()
    # end to end: row gather on the host, batch creation (plan, arena, graphs), copies, run, results
    tms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        models = ensemble.fit_rows(P.X, P.y, rows, P.op_set, P.rung, P.sis_size, P.max_dim, stream=stream)
        tms.append(time.perf_counter() - t0)
    assert [[d.ids for d in m.dims] for m in models] == [[d.ids for d in dims] for _, dims in res]
    gold = golden_fit("ensemble") or []
    parity = None
    if gold:
        eq = sum(int([d.ids for d in dims] == [g["ids"] for g in rec["dims"]]) for (_, dims), rec in zip(res, gold))
        err = max((abs(a - b) / max(abs(b), 1e-300) for (_, dims), rec in zip(res, gold)
                   for d, g in zip(dims, rec["dims"]) for a, b in zip(d.coef, g["coef"])), default=0.0)
        parity = {"tasks": len(gold), "descriptors_equal": eq, "coef_max_rel_err": err,
                  "ok": eq == len(gold) and err <= 1e-6, "tolerance_rel": 1e-6,
                  "golden": "tests/golden/ensemble_oracle.json"}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sp = oracle.Space(P.d, P.op_set, P.rung, P.grammar)
        t0 = time.perf_counter()
        for r in rows:
            oracle.fit(P.X[r], P.y[r], sp, P.sis_size, P.max_dim)
        dt = time.perf_counter() - t0
        cpu = {"value": dt, "unit": "s", "cores": cores(), "kind": "oracle",
               "sample": "all 30 models fitted by the FP64 oracle, one after another (its l0 threaded)"}
    return {"workload": P.name + ", 30 disjoint subsets of 100 samples", "metric": "time to train the ensemble",
            "unit": "ms", "launch_ms": float(np.median(ms)), "e2e_ms": 1e3 * float(np.median(tms)),
            "e2e_note": "host row gather, batch creation (plan, arena, CUDA graphs), copies, launch, results",
            "paper_seconds": {"fortran_sisso_1cpu": 182.43, "torchsisso_gpu_a100": 51.32,
                              "note": "the paper's ensemble timing table (another machine: context, not a target)"},
            "gpu_launches": 1, "cpu_baseline": cpu, "parity": parity}


def form_whitened(args):
    """Whitening (§2.4) on the workload-7 problem: N = 500, AR(1) noise and its whitening
    matrix, rung 2 (16 205 candidates), k = 10, D <= 3, FP64: time to the final descriptor,
    the whitened scoring's FP64 rate (the N x N product per candidate and step against the
    measured FP64 FMA peak), and parity with the oracle's whitened fit of the same data (the
    CPU-baseline leg)."""
    import numpy as np
    import torch
    from paper_2410_01752_gb300 import PREC_FP64, Sisso, inputs, sisso
    P = inputs.whitened_problem(0)
    stream = torch.cuda.current_stream()
    with Sisso(P.X, P.y, P.op_set, P.rung, P.sis_size, P.max_dim, precision=PREC_FP64, stream=stream,
               whiten=P.W) as s:
        s.fit()
        ms = []
        for _ in range(3):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d = s.fit()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = s.stats()
        sis_ids = [s.sis(t) for t in range(1, len(d) + 1)]
        n_feat = s.feature_count()[0]
    steps = len(d)
    flop = 2.0 * P.N * P.N * n_feat * steps           # W applied to every candidate, every step
    fp64_peak = None
    try:
        fp64_peak = sisso.measure_alu_peak(2)
    except Exception:
        pass
    rate = flop / (st["ms_screen"] / 1e3) / 1e12
    out = {"workload": P.name, "metric": "time-to-descriptor", "unit": "ms", "time_to_descriptor_ms": float(np.median(ms)),
           "descriptor": d[-1].ids, "rmse": d[-1].rmse, "gpu_launches": st["launches"],
           "whitened_scoring": {"ms_per_fit": st["ms_screen"], "flop_per_fit": flop, "tflops": rate,
                                "fp64_peak_measured_tflops": fp64_peak,
                                "frac_of_measured": rate / fp64_peak if fp64_peak else None,
                                "fp64_peak_nominal_tflops": 1.25, "frac_of_nominal": rate / 1.25,
                                "note": "2 N^2 flop per candidate and step over the whole scoring phase (raw rows, "
                                        "the FP64 product with W, whitened moments)"},
           "phase_ms": {k: st[k] for k in ("ms_screen", "ms_select", "ms_gram", "ms_l0", "ms_refit")}}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.fit(P.X, P.y, oracle.Space(P.d, P.op_set, P.rung, P.grammar), P.sis_size, P.max_dim, W=P.W)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 1e3 * dt, "unit": "ms", "cores": cores(), "kind": "oracle",
                               "sample": "the whole whitened fit by the FP64 oracle (its scoring threaded)"}
        err = max((abs(a - b) / max(abs(b), 1e-300) for g, r in zip(d, ref.dims) for a, b in zip(g.coef, r.coef)),
                  default=0.0)
        out["parity"] = {"sis_steps_equal": sis_ids == ref.sis[:len(sis_ids)],
                         "descriptors_equal": [g.ids for g in d] == [r.ids for r in ref.dims],
                         "coef_max_rel_err": err, "tolerance_rel": 1e-6,
                         "ok": sis_ids == ref.sis[:len(sis_ids)] and [g.ids for g in d] == [r.ids for r in ref.dims]
                         and err <= 1e-6}
    return out


def form_batched(args):
    """The batched multi-task form: 512 tasks in one persistent launch (CUDA graph), launch
    shape from the autotuner; every task's descriptors against the oracle's stored fits."""
    import numpy as np
    import torch
    from paper_2410_01752_gb300 import inputs, sisso
    probs = [inputs.workload5_task(p) for p in range(512)]
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    with sisso.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3, stream=stream) as b:
        tune = b.autotune(reps=1, cache_path=args.tune_cache)
        b.run(copies=False)
        ms = []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(copies=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res = b.results()
        start, end = b.timing()
        tms = []
        host = [(P.X, P.y) for P in probs]
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.load(host)
            b.run(copies=True)
            b.results()
            tms.append(time.perf_counter() - t0)
        in_bytes = sum(P.X.nbytes + P.y.nbytes for P in probs)
    gold = []
    try:
        with open(os.path.join(GOLDEN, "workload5_oracle.jsonl")) as f:
            gold = [json.loads(l) for l in f]
    except OSError:
        pass
    ok_ids, cerr = 0, 0.0
    for (st_, dims), g in zip(res, gold):
        same = st_ == 0 and [d.ids for d in dims] == [r["ids"] for r in g["dims"]]
        ok_ids += same
        if same:
            cerr = max([cerr] + [abs(a - c) / max(abs(c), 1e-300) for d, r in zip(dims, g["dims"])
                                 for a, c in zip(d.coef, r["coef"])])
    mean_ms = sum(ms) / len(ms)
    cpu = None
    if not args.no_cpu_baseline:
        r, n, dt, th = oracle_tasks_sample(probs, 5.0, seed=5)
        cpu = {"value": r, "unit": "tasks/s", "cores": th, "kind": "oracle",
               "sample": f"{n} randomly drawn tasks fitted by the FP64 oracle ({dt:.1f} s)"}
    return {"workload": BATCH_NAME.format(n=512), "metric": "tasks/s", "value": 512 / (mean_ms / 1e3),
            "unit": "tasks/s", "launch_ms": mean_ms, "tune": tune,
            "latency_ms": {"p50": float(np.percentile(end, 50)), "p99": float(np.percentile(end, 99))},
            "e2e": {"value": 512 / (sum(tms) / len(tms)), "unit": "tasks/s", "h2d_bytes_per_step": int(in_bytes),
                    "d2h_bytes_per_step": int(512 * sisso.C.sizeof(sisso.TaskResult))},
            "gpu_launches": 1, "cpu_baseline": cpu,
            "parity": {"tasks": len(gold), "descriptors_equal": ok_ids, "coef_max_rel_err": cerr,
                       "ok": len(gold) == 512 and ok_ids == 512 and cerr <= 1e-6, "tolerance_rel": 1e-6}}


def form_learned(args):
    """The learned proposal: trained on the method's own exhaustive results (2000 problems),
    then the fit's time to the D = 5 descriptor with and without it on held-out problems,
    judged by the oracle's stored exhaustive fits."""
    import numpy as np
    from paper_2410_01752_gb300 import inputs, proposal, sisso
    t0 = time.perf_counter()
    X, t = proposal.training_set(2000, k=60, per_problem=768, top=256, seed=0)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, rel_loss = proposal.train(X, t, seed=0, epochs=10, batch=2048, lr=1e-3)
    t_train = time.perf_counter() - t0
    gold = golden_fit("workload4") or []
    probs = [inputs.workload4(r["p"], held_out=True) for r in gold]
    proposal.evaluate(net, probs[:1], frac=0.01)
    res = proposal.evaluate(net, probs, frac=0.01)
    zero = sisso.MLP(0)
    zero.set_params(np.zeros(sisso.MLP_PARAMS, dtype=np.float32))
    res0 = proposal.evaluate(zero, probs, frac=0.01)
    ok = [(r, g, r0) for r, g, r0 in zip(res, gold, res0) if "recall" in r]
    match = [r["learned_ids"] == g["dims"][-1]["ids"] for r, g, _ in ok]
    plain_match = [r["plain_ids"] == g["dims"][-1]["ids"] for r, g, _ in ok]
    cert_match = [r["certified_ids"] == g["dims"][-1]["ids"] for r, g, _ in ok]
    ms_l = float(np.mean([r["fit_learned_ms_device"] for r, _, _ in ok])) if ok else None
    ms_p = float(np.mean([r["fit_plain_ms_device"] for r, _, _ in ok])) if ok else None
    ms_c = float(np.mean([r["fit_certified_ms_device"] for r, _, _ in ok])) if ok else None
    cpu = None
    if not args.no_cpu_baseline and probs:
        import oracle
        P = probs[0]
        c = sisso.Sisso(P.X, P.y, P.op_set, P.rung, 60, 5, grammar=P.grammar)
        c.fit()
        S = sum((c.sis(t) for t in range(1, 6)), [])[:60]
        G, b, syy = c.subspace_gram(S)
        c.close()
        t0 = time.perf_counter()
        _, _, ex = oracle.l0(G, b, syy, P.N, 5, S, nthreads=cores())
        dt = time.perf_counter() - t0
        cpu = {"value": ex / dt, "unit": "subsets/s", "cores": cores(), "kind": "oracle",
               "sample": f"exhaustive D = 5 over the first 60 screened features: C(60,5) = {ex} subsets ({dt:.1f} s)"}
    return {"workload": "learned proposal: D=5 over 300 features (k=60), held-out problems of the stored oracle fits",
            "metric": "time-to-descriptor vs plain at equal RMSE", "unit": "ms",
            "fit_learned_ms": ms_l, "fit_plain_ms": ms_p, "speedup_vs_plain": (ms_p / ms_l) if ok else None,
            "fit_certified_ms": ms_c, "certified_speedup_vs_plain": (ms_p / ms_c) if ok else None,
            "certified_equals_oracle": sum(cert_match),
            "certified_prefixes_mean": float(np.mean([r["certified_prefixes"] for r, _, _ in ok])) if ok else None,
            "problems": len(ok), "learned_equals_oracle": sum(match), "plain_equals_oracle": sum(plain_match),
            "greedy_only_equals_exhaustive": sum(r0["recall"] for _, _, r0 in ok),
            "trained_equals_exhaustive": sum(r["recall"] for r, _, _ in ok),
            "training": {"problems": 2000, "examples": int(X.shape[0]), "data_s": t_data, "train_s": t_train,
                         "loss_rel_to_target_var": rel_loss},
            "gpu_launches": int(round(float(np.mean([r["fit_learned_launches"] for r, _, _ in ok])))) if ok else None,
            "cpu_baseline": cpu,
            "parity": {"ok": bool(ok) and all(cert_match),
                       "note": "final D = 5 descriptor of the certified learned fit vs the oracle (the uncertified "
                               "fit's matches are learned_equals_oracle)"}}


def workload2_config(P, n_features: int, world: int = 1):
    """The default line's config (both arms print the same dict)."""
    return {"workload": P.name, "N": P.N, "d": P.d, "rung": P.rung, "grammar": "new_x_prev",
            "sis_size": P.sis_size, "max_dim": P.max_dim, "n_features": int(n_features),
            "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"}


def run_reference(args, rank: int):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    import oracle
    from paper_2410_01752_gb300 import inputs
    if rank != 0:
        return
    P = inputs.workload2(0)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline_sample(P, per_step / 4, seed=1)
    rates, dts, samples = [], [], []
    for k in range(args.steps):
        r, m, dt, th = cpu_baseline_sample(P, per_step, seed=100 + k)
        rates.append(r)
        dts.append(dt)
        samples.append(m)
    value = sum(samples) / sum(dts)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload2_config(P, oracle.Space(P.d, P.op_set, P.rung, P.grammar).n_features, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                         "sample": f"{samples[0]} random candidate ids per step scored in FP64 over all {P.N} samples"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_mixed(args):
    """Mixed-precision forms vs the plain FP32 form: time to the final descriptor, equal
    descriptor and RMSE, errors against the oracle's stored FP64 fit."""
    import numpy as np
    import torch
    from paper_2410_01752_gb300 import PREC_FP32, PREC_MIXED_BF16, PREC_MIXED_FP16, Sisso, build, inputs
    build.build()
    torch.cuda.set_device(0)
    P = inputs.workload3(0)
    Xd, yd = torch.from_numpy(P.X).cuda(), torch.from_numpy(P.y).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    res = {}
    for name, prec, gram in (("plain_fp32", PREC_FP32, 0), ("fp32_tf32x3_gram", PREC_FP32, 2),
                             ("mixed_bf16", PREC_MIXED_BF16, 0), ("mixed_fp16", PREC_MIXED_FP16, 0)):
        s = Sisso(Xd, yd, P.op_set, P.rung, P.sis_size, P.max_dim, precision=prec, grammar=P.grammar, stream=stream,
                  gram=gram)
        for _ in range(args.warmup):
            s.fit()
        ms, st = [], None
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d = s.fit()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = s.stats()
        S_all = sum((s.sis(t) for t in range(1, len(d) + 1)), [])
        res[name] = {"ms": sum(ms) / len(ms), "desc": d[-1], "S": S_all, "stats": st}
        s.close()
    plain = res["plain_fp32"]
    # the oracle's stored FP64 fit of the same problem (tests/golden/workload3_oracle.json,
    # written from the oracle alone): its final descriptor, coefficients and RMSE
    rec = (golden_fit("workload3") or [None])[0]
    ref = rec["dims"][-1] if rec else None
    out = {}
    for name, r in res.items():
        d = r["desc"]
        same = ref is not None and d.ids == ref["ids"]
        out[name] = {
            "time_to_descriptor_ms": r["ms"], "descriptor": d.ids, "rmse": d.rmse,
            "same_descriptor_as_oracle": same, "same_subspace_as_plain": r["S"] == plain["S"],
            "coef_rel_err_vs_oracle": [abs(a - b) / max(abs(b), 1e-300) for a, b in zip(d.coef, ref["coef"])] if same else None,
            "rmse_rel_err_vs_oracle": abs(d.rmse - ref["rmse"]) / ref["rmse"] if ref else None,
            "rmse_rel_diff_vs_plain": abs(d.rmse - plain["desc"].rmse) / plain["desc"].rmse,
            "ms_gram": r["stats"]["ms_gram"], "ms_l0": r["stats"]["ms_l0"], "ms_refit": r["stats"]["ms_refit"],
            "ms_screen_pair": r["stats"]["ms_screen_pair"], "screen_tensor_cores": bool(r["stats"]["screen_tc"]),
            "subsets_refit": r["stats"]["subsets_refit"]}
    m = out["mixed_bf16"]
    line = {
        "metric": "time-to-descriptor vs plain at equal RMSE", "value": m["time_to_descriptor_ms"] / 1e3, "unit": "s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["time_to_descriptor_ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": P.name, "N": P.N, "d": P.d, "rung": P.rung, "sis_size": P.sis_size,
                   "max_dim": P.max_dim, "l2": "flushed between steps (256 MB write)"},
        "speedup_vs_plain": {k: out["plain_fp32"]["time_to_descriptor_ms"] / v["time_to_descriptor_ms"]
                             for k, v in out.items() if k != "plain_fp32"},
        "forms": out, "oracle_reference": {"golden": "tests/golden/workload3_oracle.json",
                                           "ids": ref["ids"], "coef": ref["coef"], "rmse": ref["rmse"]} if ref else None,
    }
    print(json.dumps(line), flush=True)


def batch_flops(probs, res) -> float:
    """Algorithmic FP32 flops of the batched workload's screening: FP32_FLOP_PER_CAND_SAMPLE
    per candidate and sample of each task's space, for every screening step it ran."""
    import oracle
    tot = 0.0
    for P, (_, dims) in zip(probs, res):
        tot += oracle.Space(P.d, P.op_set, P.rung, P.grammar).n_features * P.X.shape[0] * max(len(dims), 1)
    return tot * FP32_FLOP_PER_CAND_SAMPLE


def oracle_tasks_sample(probs, seconds: float, seed: int = 0):
    """The FP64 oracle fitting randomly drawn tasks of the batch on all host cores for about
    `seconds`; returns (tasks/s, tasks fitted, wall seconds, threads)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    th = cores()
    done, t0 = 0, time.perf_counter()
    while True:
        P = probs[int(rng.integers(0, len(probs)))]
        oracle.fit(P.X, P.y, oracle.Space(P.d, P.op_set, P.rung, P.grammar), P.sis_size, P.max_dim, nthreads=th)
        done += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            return done / dt, done, dt, th


BATCH_NAME = "batched multi-task: {n} tasks, N~U{{20..2000}}, d~U{{4..12}}, x~U[0.5,5], rung 2, 9 ops, k=50, D<=3"


def run_batch(args, rank: int):
    """Batched multi-task workload: every task in one persistent launch (CUDA graph)."""
    import numpy as np
    from paper_2410_01752_gb300 import inputs
    probs = [inputs.workload5_task(p) for p in range(args.tasks)]
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
        for k in range(args.warmup):
            oracle_tasks_sample(probs, per_step / 4, seed=k)
        done, dts = 0, 0.0
        th = cores()
        for k in range(args.steps):
            _, n, dt, th = oracle_tasks_sample(probs, per_step, seed=100 + k)
            done += n
            dts += dt
        value = done / dts
        line = {"impl": "reference", "metric": "tasks/s", "value": value, "unit": "tasks/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dts / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": BATCH_NAME.format(n=args.tasks), "tasks": args.tasks},
                "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": th, "kind": "oracle",
                                 "sample": f"{done} randomly drawn tasks fitted by the FP64 oracle"},
                "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import torch
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    b = sisso.Batch([(P.X, P.y) for P in probs], probs[0].op_set, 2, 50, 3, stream=stream)
    tune = b.get_tune() if args.no_autotune else b.autotune(reps=2, cache_path=args.tune_cache)
    for _ in range(args.warmup):
        b.run(copies=False)
    ms, stats = [], []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(copies=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            stats.append(b.stats())
    res = b.results()
    start, end = b.timing()
    failed = sum(1 for st_, _ in res if st_ != 0)
    mean_ms = sum(ms) / len(ms)
    value = args.tasks / (mean_ms / 1e3)
    # end to end through the C ABI: new host inputs into the pinned staging buffer, one graph
    # launch with the copies, results read back
    e2e = None
    if not args.no_e2e:
        host = [(P.X.copy(), P.y.copy()) for P in probs]
        in_bytes = sum(X.nbytes + y.nbytes for X, y in host)
        tms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.load(host)
            b.run(copies=True)
            r2 = b.results()
            tms.append(time.perf_counter() - t0)
        assert [d.ids for _, dd in r2 for d in dd] == [d.ids for _, dd in res for d in dd]
        e2e = {"value": args.tasks / (sum(tms) / len(tms)), "unit": "tasks/s", "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": int(args.tasks * sisso.C.sizeof(sisso.TaskResult))}
    flop = batch_flops(probs, res)
    pk = peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = alu_peak(sms, mhz)["peak"]
    achieved = flop / (mean_ms / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "k_batch (persistent, all stages)", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": captured_batch_traffic(tune),
            "peak_source": alu_peak(sms, mhz)["source"],
            "flop_per_launch": flop, "launch_ms": mean_ms,
            "algorithmic_unit": f"{FP32_FLOP_PER_CAND_SAMPLE} flop per candidate-sample of screening, every task and step run",
            "score_stage_frac": None}
    cpu = None
    if not args.no_cpu_baseline:
        r, n, dt, th = oracle_tasks_sample(probs, args.cpu_seconds)
        cpu = {"value": r, "unit": "tasks/s", "cores": th, "kind": "oracle",
               "sample": f"{n} randomly drawn tasks of the batch fitted by the FP64 oracle ({dt:.1f} s)"}
    st = stats[-1]
    # the screening stage alone: its flops over its share of the SMs' time (CTA-time / CTAs per SM)
    score_sm_s = st["stage_ms"][3] / 1e3 / (st["grid"] / sms)
    roof["score_stage_frac"] = flop / (score_sm_s / sms) / 1e12 / peak if score_sm_s > 0 else None
    names = ["-", "start", "level", "score", "gram", "bound", "band", "flat", "select", "refit", "idle", "opsum",
             "select.radix", "select.rescore", "select.sort", "select.walk"]
    line = {
        "metric": "tasks/s", "value": value, "unit": "tasks/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_NAME.format(n=args.tasks), "tasks": args.tasks, "tune": tune,
                   "l2": "flushed between steps (256 MB write)", "graph": "one persistent launch per step"},
        "latency_ms": {"p50": float(np.percentile(end, 50)), "p99": float(np.percentile(end, 99)),
                       "max": float(end.max()), "note": "per task, from the launch's first CTA to its last result"},
        "service_ms": {"p50": float(np.percentile(end - start, 50)), "p99": float(np.percentile(end - start, 99))},
        "tasks_failed": failed,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 1,
        "clocks": clk.summary(),
        "stage_cta_ms": {names[q]: st["stage_ms"][q] for q in range(16) if names[q] != "-"},
        "subsets_fit": st["subsets_fit"], "subsets_refit": st["subsets_refit"],
        "windows_grown": st["windows_grown"], "windows_saturated": st["windows_saturated"],
        "walk_visits": st["walk_visits"], "grid": st["grid"],
    }
    print(json.dumps(line), flush=True)
    b.close()


def learned_oracle_parity(res):
    """The held-out problems with stored oracle fits (tests/golden/workload4_oracle.json):
    how many of the plain, learned and certified D = 5 descriptors equal the oracle's."""
    gold = golden_fit("workload4") or []
    pairs = [(r, g) for r, g in zip(res, gold) if "recall" in r]
    if not pairs:
        return None
    want = [g["dims"][-1]["ids"] for _, g in pairs]
    return {"problems": len(pairs), "golden": "tests/golden/workload4_oracle.json",
            "plain_equals_oracle": sum(r["plain_ids"] == w for (r, _), w in zip(pairs, want)),
            "learned_equals_oracle": sum(r["learned_ids"] == w for (r, _), w in zip(pairs, want)),
            "certified_equals_oracle": sum(r["certified_ids"] == w for (r, _), w in zip(pairs, want))}


def run_learned(args):
    """Learned proposal: train the network on the method's own exhaustive results, then on
    held-out problems compare the fit's time to the D = 5 descriptor with and without it;
    the exhaustive search judges recall, and the oracle's stored fits judge the first eight."""
    import numpy as np
    import torch
    from paper_2410_01752_gb300 import build, inputs, proposal, sisso
    build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    X, t = proposal.training_set(args.train_problems, k=60, per_problem=768, top=256, seed=0)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, rel_loss = proposal.train(X, t, seed=0, epochs=10, batch=2048, lr=1e-3)
    t_train = time.perf_counter() - t0
    zero = sisso.MLP(0)
    zero.set_params(np.zeros(sisso.MLP_PARAMS, dtype=np.float32))
    untrained = sisso.MLP(0)
    probs = [inputs.workload4(p, held_out=True) for p in range(args.eval_problems)]
    for _ in range(args.warmup):
        proposal.evaluate(net, probs[:1], frac=args.frac)
    res = proposal.evaluate(net, probs, frac=args.frac)
    ok = [r for r in res if "recall" in r]
    others = {}
    n_cmp = min(len(probs), 32)
    for name, m in (("greedy_only", zero), ("untrained", untrained)):
        rr = [r for r in proposal.evaluate(m, probs[:n_cmp], frac=args.frac) if "recall" in r]
        others[name] = {"recall": sum(r["recall"] for r in rr) / max(len(rr), 1), "problems": len(rr)}
    first = {P.name for P in probs[:n_cmp]}
    trained_first = [r for r in ok if r["name"] in first]
    ms_l = float(np.mean([r["fit_learned_ms_device"] for r in ok]))
    ms_p = float(np.mean([r["fit_plain_ms_device"] for r in ok]))
    ms_c = float(np.mean([r["fit_certified_ms_device"] for r in ok]))
    recall = sum(r["recall"] for r in ok) / max(len(ok), 1)
    same = sum(r["same_descriptor"] and r["rmse_rel_diff"] <= 1e-5 for r in ok) / max(len(ok), 1)
    line = {
        "metric": "time-to-descriptor vs plain at equal RMSE", "value": ms_l / 1e3, "unit": "s",
        "n_gpus": 1, "steps": len(ok), "warmup": args.warmup, "ms_per_step": ms_l, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
        "config": {"workload": "learned proposal: D=5 over 300 features (k=60, 5 SIS steps), N~U{500..2000}, "
                               "d~U{8..12}, x~U[1,5], 3-5 planted rung-2 terms",
                   "train_problems": args.train_problems, "eval_problems": len(ok), "frac": args.frac,
                   "train_examples": int(X.shape[0])},
        "plain_ms": ms_p, "speedup_vs_plain": ms_p / ms_l,
        "certified_ms": ms_c, "certified_speedup_vs_plain": ms_p / ms_c,
        "certified_same_descriptor": sum(r["certified_ids"] == r["plain_ids"] for r in ok) / max(len(ok), 1),
        "recall": recall, "same_descriptor_equal_rmse": same,
        "oracle_parity": learned_oracle_parity(res),
        "recall_first_n": {"trained": sum(r["recall"] for r in trained_first) / max(len(trained_first), 1),
                           **{k: v["recall"] for k, v in others.items()}, "problems": n_cmp},
        "l0_d5_ms": {"exhaustive": 1e3 * float(np.mean([r["exhaustive_s"] for r in ok])),
                     "learned": 1e3 * float(np.mean([r["learned_s"] for r in ok]))},
        "subsets_solved": {"exhaustive": ok[0]["examined_exhaustive"] if ok else None,
                           "learned_mean": float(np.mean([r["examined_learned"] for r in ok])) if ok else None},
        "training": {"data_s": t_data, "train_s": t_train, "loss_rel_to_target_var": rel_loss},
        "gpu_launches": int(round(float(np.mean([r["fit_learned_launches"] for r in ok])))) if ok else None,
        "gpu_launches_note": "kernel launches of one learned fit (mean over the held-out problems)",
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == 3:
        run_mixed(args)
        return
    if args.workload == 4:
        run_learned(args)
        return
    if args.workload == 5:
        run_batch(args, int(os.environ.get("RANK", "0")))
        return
    if args.workload == 7:         # whitening (§2.4): the form on its own line
        import torch
        from paper_2410_01752_gb300 import build
        build.build()
        torch.cuda.set_device(0)
        print(json.dumps(form_whitened(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        import oracle
        oracle.build()
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_2410_01752_gb300 import PREC_FP32, Sisso, build, inputs

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        build.build()
    P = inputs.workload2(rank, N=args.N, d=args.d)
    Xd = torch.from_numpy(P.X).cuda()
    yd = torch.from_numpy(P.y).cuda()
    stream = torch.cuda.current_stream()
    s = Sisso(Xd, yd, P.op_set, P.rung, P.sis_size, P.max_dim, precision=PREC_FP32, grammar=P.grammar,
              stream=stream, device=local)
    n_feat, sizes = s.feature_count()
    sizes = sizes[: P.rung + 1]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    for _ in range(args.warmup):
        s.fit()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    step_ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            desc = s.fit()
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            step_ms.append(e0.elapsed_time(e1))
            stats.append(s.stats())
    total_ms = sum(step_ms)
    cand = sum(st["candidates_scored"] for st in stats)
    subsets = sum(st["subsets_fit"] for st in stats)
    launches = sum(st["launches"] for st in stats)
    total_ms, (cand, subsets, launches) = job_totals(total_ms, [cand, subsets, launches], dist, "cuda")
    value = cand / (total_ms / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e, e2e_step_s = None, None
    if not args.no_e2e:
        Xh = torch.from_numpy(P.X).pin_memory()
        yh = torch.from_numpy(P.y).pin_memory()
        e2e_ms, e2e_cand, d2h = [], 0, 0
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            with Sisso(Xh.numpy(), yh.numpy(), P.op_set, P.rung, P.sis_size, P.max_dim, precision=PREC_FP32,
                       grammar=P.grammar, device=local) as se:
                dd = se.fit()
                e2e_cand += se.stats()["candidates_scored"]
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            d2h = sum(8 * len(x.ids) + 8 * len(x.coef) + 16 for x in dd)
        tot, (e2e_cand,) = job_totals(sum(e2e_ms), [e2e_cand], dist, "cuda")
        e2e_step_s = tot / args.steps / 1e3
        e2e = {"value": e2e_cand / (tot / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(P.X.nbytes + P.y.nbytes),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (the fused pair kernel), timed with CUDA events on
    # its launch stream inside the library
    pair_ms = sum(st["ms_screen_pair"] for st in stats)
    pair_launches = sum(st["screen_pair_launches"] for st in stats)
    n_unary = sum(1 for b in range(4, 12) if P.op_set >> b & 1)
    cand_pair = top_binary_candidates(sizes, n_unary)
    flop_launch = cand_pair * P.N * FP32_FLOP_PER_CAND_SAMPLE
    avg_launch_s = (pair_ms / max(pair_launches, 1)) / 1e3
    achieved = flop_launch / avg_launch_s / 1e12
    pk = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    apk = alu_peak(sms, mhz)
    peak = apk["peak"]
    full_size = (P.N, P.d) == (1000, 10)
    roof = {"bound": "alu", "kernel": "k_score_pairs<float>", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": captured_traffic() if full_size else None,
            "peak_source": apk["source"], "fp32_measured_tflops": max(apk.get("fp32", 0.0), apk.get("fp32x2", 0.0)),
            "frac_of_measured": achieved / max(apk.get("fp32", 0.0), apk.get("fp32x2", 0.0), 1e-9),
            "fp64_measured_tflops": apk.get("fp64"),
            "flop_per_launch": flop_launch, "launch_ms": avg_launch_s * 1e3,
            "algorithmic_unit": f"{FP32_FLOP_PER_CAND_SAMPLE} flop per candidate-sample x {cand_pair} candidates x {P.N} samples"}

    cpu = None
    if not args.no_cpu_baseline:
        r, m, dt, th = cpu_baseline_sample(P, args.cpu_seconds)
        r1, m1, dt1, _ = cpu_baseline_sample(P, max(1.0, args.cpu_seconds / 4), seed=1, threads=1)
        cpu = {"value": r, "unit": UNIT, "cores": th, "kind": "oracle",
               "sample": f"{m} random candidate ids of the workload scored in FP64 over all {P.N} samples ({dt:.1f} s)",
               "value_1thread": r1, "sample_1thread": f"{m1} random candidate ids on one thread ({dt1:.1f} s)"}

    # parity of the timed fit with the oracle's stored fit of the same problem
    parity = None
    rec = golden_fit("workload2") if (P.N, P.d) == (1000, 10) and rank == 0 else None
    if rec:
        parity = compare_fit([s.sis(t) for t in range(1, len(desc) + 1)], desc, rec[0], 1e-6)
        parity["golden"] = "tests/golden/workload2_oracle.json"
    l0_roof = l0_roofline(s, len(desc), peak, sms, mhz) if len(desc) >= 3 else None
    forms = None
    if not args.no_forms and world == 1:
        forms = {"mixed_precision": form_mixed(args), "batched": form_batched(args),
                 "learned_proposal": form_learned(args), "ensemble": form_ensemble(args),
                 "whitened": form_whitened(args)}

    d_last = desc[-1] if desc else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload2_config(P, n_feat, world),
        "parity": parity,
        "l0_subsets_fit_per_s": subsets / (sum(st["ms_l0"] for st in stats) / 1e3),
        "l0_subsets_fit_per_s_note": "subsets of every step's search / the searches' device time (ms_l0)",
        "time_to_descriptor_s": total_ms / args.steps / 1e3,
        "time_to_descriptor_e2e_s": e2e_step_s,
        "time_to_descriptor_e2e_note": "one fit through the C ABI from host buffers, context creation included",
        "l0_roofline": l0_roof,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "phase_ms": {k: sum(st[k] for st in stats) / args.steps for k in
                     ("ms_screen", "ms_screen_pair", "ms_select", "ms_radix", "ms_rescore", "ms_sort", "ms_walk",
                      "ms_gram", "ms_l0", "ms_refit", "ms_fit", "walk_visited", "walk_dup_checks")},
        "descriptor": {"ids": d_last.ids, "coef": d_last.coef, "rmse": d_last.rmse, "r2": d_last.r2,
                       "expr": [s.expr(i) for i in d_last.ids]} if d_last else None,
        "window_grown": sum(st["window_grown"] for st in stats),
        "window_saturated": max(st["window_saturated"] for st in stats),
        "pm_keys_direct_per_fit": sum(st["pm_keys_direct"] for st in stats) / args.steps,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
