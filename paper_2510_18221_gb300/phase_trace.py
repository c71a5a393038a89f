"""Phase split of the persistent environment kernel on the GPU.

Runs a named workload, switches on the kernel's phase trace
(eco_trace_phases) for up to 64 steps and prints, per grid barrier, when
the last CTA arrived and when CTA 0 passed it, and when the last CTA ended,
in microseconds from CTA 0's start (median, min and max over the steps;
steps with and without birth claimants apart for the end).

    python -m paper_2510_18221_gb300.phase_trace [--workload paper|batched|...]
        [--precision bf16] [--warmup 5] [--steps 60] [--json]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

TR_START, TR_ARRIVE0, TR_PASS0, TR_END, TR_STEP, TR_CLAIMANTS, TR_BARRIERS = 0, 1, 5, 9, 10, 11, 12


def summarise(rows: np.ndarray) -> dict:
    """Per-barrier arrival / pass and end times (us from CTA 0's start) of
    the traced rows of an eco_read_phase_trace table."""
    rows = rows[rows[:, TR_START] > 0].astype(np.int64)
    out = {"steps": int(len(rows))}
    if len(rows) == 0:
        return out
    t0 = rows[:, TR_START]

    def stat(v):
        v = np.asarray(v, dtype=float) / 1e3
        return {"median": float(np.median(v)), "min": float(v.min()), "max": float(v.max())}

    nbar = int(rows[:, TR_BARRIERS].min())
    for k in range(nbar):
        out["arrive_%d" % k] = stat(rows[:, TR_ARRIVE0 + k] - t0)
        out["pass_%d" % k] = stat(rows[:, TR_PASS0 + k] - t0)
    out["end"] = stat(rows[:, TR_END] - t0)
    births = rows[:, TR_CLAIMANTS] > 0
    if births.any():
        out["end_with_claimants"] = stat(rows[births, TR_END] - t0[births])
    if (~births).any():
        out["end_without_claimants"] = stat(rows[~births, TR_END] - t0[~births])
    out["claimants_median"] = float(np.median(rows[:, TR_CLAIMANTS]))
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--json", action="store_true")
    args = ap.parse_args()

    import torch

    from . import eco, workloads

    over = {} if args.precision is None else {"precision": args.precision}
    if args.workload == "batched":
        # the 64 uneven worlds of the batched workload, in one handle
        envs = workloads.batched(64, **over)
        w = {"name": "batched-64worlds-%s" % envs[0]["precision"]}
    else:
        envs = w = workloads.get(args.workload, **over)
    env = eco.Env(envs)
    try:
        env.reset()
        env.prepare()
        env.step(args.warmup)
        env.trace_phases(True)
        env.step(min(args.steps, eco.ECO_TRACE_STEPS))
        torch.cuda.synchronize()
        rows = env.phase_trace()
        env.trace_phases(False)
    finally:
        env.close()
    res = summarise(rows)
    name = w["name"]
    if args.precision is not None and name.rsplit("-", 1)[-1] in ("fp32", "bf16", "fp8"):
        name = name.rsplit("-", 1)[0] + "-" + args.precision
    res["workload"] = name
    if args.json:
        print(json.dumps(res))
        return
    print("%s: %d traced steps, median claimants %.0f (us from CTA 0's start)"
          % (name, res["steps"], res.get("claimants_median", 0)))
    for k, v in res.items():
        if isinstance(v, dict):
            print("  %-22s median %7.2f  min %7.2f  max %7.2f" % (k, v["median"], v["min"], v["max"]))


if __name__ == "__main__":
    main()
