#!/usr/bin/env python3
"""Throughput of the full environment step (policy + environment) on GB300.

Metric: agent-steps per second -- the number of agents alive at the start
of each step, summed over the timed steps, divided by the device time of
those steps -- plus the HBM bandwidth the policy kernel achieves against
the measured copy bandwidth of this GPU.

Default workload: one 1024x1024 world, 65,536 agent slots, 50,000 founders,
per-agent MLP 371 -> 64 -> 64 -> 9 with weights streamed as BF16 (FP32
accumulation), rules of the mid-scale workload.  The weight stream of one
step (~2.9 GB) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl eco|reference]

With N > 1 (launched by torch.distributed.run) every rank advances its own
independent world (seed + rank) on its own GPU: weak scaling, no collective
on the data path; the timing is the maximum over ranks.  --impl reference
times the CPU oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-steps/sec at 65,536 agents (policy+env) and policy-kernel HBM GB/s vs peak"
UNIT = "agent-steps/s"
# Kernels per step: the policy kernel (with the move claims) plus either one
# persistent kernel for every environment phase, or one kernel per phase:
# move+eat+attack claims, attack transfer+metabolism+death, birth claim,
# birth assign, mutate, regrow, finish, and the alive list.
KERNELS_PER_STEP = {0: 2, 1: 9}


def kernels_per_step(launch_mode, rules):
    """Library kernels per step; the per-phase form of the terrain rules
    adds the two passes of the water flow."""
    return KERNELS_PER_STEP[launch_mode] + (2 if launch_mode == 1 and rules == "terrain" else 0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="eco", choices=["eco", "reference"])
    ap.add_argument("--workload", default="paper")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU time budget of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp8"],
                    help="override the workload's streamed weight precision")
    ap.add_argument("--side", type=int, default=None,
                    help="a smaller world of the same workload (with --slots and --founders), "
                         "e.g. for a profiler capture")
    ap.add_argument("--slots", type=int, default=None)
    ap.add_argument("--founders", type=int, default=None)
    ap.add_argument("--policy-variant", type=int, default=0,
                    help="force a policy-kernel variant (0: autotune)")
    ap.add_argument("--launch-mode", type=int, default=0, choices=[0, 1],
                    help="environment phases: 0 persistent kernel, 1 one kernel per phase")
    args = ap.parse_args()
    scale = (args.side, args.slots, args.founders)
    if any(v is not None for v in scale) and not all(v is not None for v in scale):
        ap.error("--side, --slots and --founders go together")
    return args


def reduce_over_ranks(dist, times, counts, device="cpu"):
    """Whole-job figures across ranks: the maximum of each time (the job
    ends when the slowest rank ends) and the sum of each count (agent-steps
    of every rank's world).  Returns the times, then the counts."""
    import torch
    t = torch.tensor([float(v) for v in times], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()] + [int(v) for v in c.tolist()]


def make_workloads(args, rank):
    """The worlds one rank advances: one named workload, or the 64 uneven
    worlds of the batched workload (seeds offset per rank)."""
    from paper_2510_18221_gb300 import workloads
    if args.workload == "batched":
        envs = workloads.batched(64, seed=0, base_seed=1000 * rank,
                                 precision=args.precision or "bf16")
    else:
        base = workloads.get(args.workload)
        if args.side is not None:
            envs = [workloads.scaled(args.workload, args.side, args.slots, args.founders,
                                     seed=base["seed"] + rank)]
        else:
            envs = [workloads.get(args.workload, seed=base["seed"] + rank)]
        if args.precision:
            envs[0]["precision"] = args.precision
            head, _, last = envs[0]["name"].rpartition("-")
            envs[0]["name"] = (head if last in ("fp32", "bf16", "fp8") else envs[0]["name"]) + \
                "-" + args.precision
    return envs


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def committed_traffic(workload_name):
    """Per-launch DRAM bytes of the policy kernel from a committed ncu
    summary, if one exists for this workload and the current kernel."""
    path = os.path.join(ROOT, "profiles", "policy_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    rec = d.get(workload_name)
    if not rec:
        return None
    return rec


class ClockSampler:
    """nvidia-smi clock / throttle sampling around the timed region.  Each
    sample carries nvidia-smi's own timestamp; `stop(t0, t1)` keeps the
    samples whose timestamp lies in the wall-clock window [t0, t1] of the
    timed region, and falls back to the samples nearest to it (flagged
    "window": "adjacent") when the region is shorter than the interval."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, device_id: str | None):
        self.lines = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", str(self.INTERVAL_MS)]
        if device_id:
            cmd += ["-i", device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.5)   # nvidia-smi start-up, so that sampling covers the region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    @staticmethod
    def _when(stamp: str):
        import datetime
        try:
            return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t0: float, t1: float, t2: float | None = None):
        """Summary of the samples of the timed region [t0, t1].  A region
        shorter than a few sampling intervals holds too few samples; then
        the samples of [t0, t2] are used -- the timed region and the
        passes that follow it back to back on the same GPU (policy timing,
        end to end) -- and "window" says so."""
        if not self.proc:
            return None
        time.sleep(2 * self.INTERVAL_MS / 1000.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                power = float(parts[4]) if parts[4] not in ("", "[N/A]") else None
                rows.append((self._when(parts[0]), float(parts[2]), float(parts[3]), parts[6:10], power))
            except ValueError:
                continue
        inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        window = "timed region"
        if len(inside) < 3 and t2 is not None:
            inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t2]
            window = "timed region + the timing and end-to-end passes after it (%.2f s)" % (t2 - t0)
        if not inside:
            timed = [r for r in rows if r[0] is not None]
            timed.sort(key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))
            inside = timed[:2]
            window = "adjacent"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for r in inside:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": sorted(reasons),
                "samples": len(inside), "interval_ms": self.INTERVAL_MS, "window": window,
                "power_w_max": max((r[4] for r in inside if r[4] is not None), default=None)}


def mlp_shape(w) -> str:
    """Layer widths of the policy: input, H per hidden activation, actions."""
    layers = w.get("n_hidden", 1) if w.get("policy_form", "plain") == "paper" else 1
    nch = 4 if w.get("rules") == "terrain" else 3     # terrain: + elevation channel
    return "-".join(str(v) for v in [nch * w["patch_k"] ** 2 + w["n_scalars"]]
                    + [w["hidden"]] * (1 + layers) + [w["n_actions"]])


def cpu_baseline_sample(w, seconds, window, steps_cap=None):
    """Time the CPU oracle on a bounded sample of the workload: the same MLP,
    rules and precision on a 256x256 world with the same founder density
    (4,096 slots, 3,125 founders), stepping through the same post-reset
    window (w0, w1) as the GPU measurement; the world is reset (untimed)
    whenever the window is exhausted, until `seconds` of stepping (or
    `steps_cap` timed steps) have been spent."""
    import oracle
    side = 256
    scale = (side * side) / float(w["side"] * w["side"])
    founders = max(1, int(round(w["init_alive"] * scale)))
    slots = max(founders, int(round(w["slots"] * scale)))
    sw = dict(w, side=side, slots=slots, init_alive=founders,
              name="%s sample %dx%d %d slots" % (w["name"], side, side, slots))
    o = oracle.Oracle(sw)
    w0, w1 = window
    agent_steps, n, el = 0, 0, 0.0
    while True:
        o.reset()
        for _ in range(w0):
            o.step_once()
        for _ in range(w0, w1):
            t0 = time.perf_counter()
            _, st, _ = o.step_once()
            el += time.perf_counter() - t0
            agent_steps += st["agent_steps"]
            n += 1
            if (steps_cap is None and el >= seconds and n >= 2) or (steps_cap is not None and n >= steps_cap):
                break
        else:
            continue
        break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": agent_steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d timed steps (within steps %d..%d after reset) of a %dx%d world, %d slots, "
                      "%d founders, MLP %s %s (same rules and founder density), %.1f s" %
                      (n, w0, w1, side, side, slots, founders, mlp_shape(w), w["precision"], el)}, \
        agent_steps, el


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2510_18221_gb300 import workloads
    w = workloads.get(args.workload)
    # K timed oracle steps on the bounded sample, after W untimed ones
    window = (args.warmup, args.warmup + args.steps)
    rec, agent_steps, el = cpu_baseline_sample(w, 0, window, steps_cap=max(1, args.steps))
    value = agent_steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "sample": rec["sample"]},
            "cpu_baseline": dict(rec, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    from paper_2510_18221_gb300 import eco, workloads

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    envs = make_workloads(args, rank)
    w = envs[0]
    env = eco.Env(envs, policy_variant=args.policy_variant, launch_mode=args.launch_mode)

    def agent_steps_of(stats):
        return sum(s["agent_steps"] for s in stats)

    # ---- device-timed region -------------------------------------------------
    env.reset()
    env.prepare()                    # autotunes the policy kernel, builds the step graphs
    env.step(args.warmup)
    torch.cuda.synchronize()
    s0 = env.stats()
    props = torch.cuda.get_device_properties(local)
    dev_id = None
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        dev_id = "GPU-" + str(uuid)
    clocks = ClockSampler(dev_id) if rank == 0 else None
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    # eco_step_timed: graphs of 8 steps, the first step's policy kernel of
    # each between two CUDA-event records on the library stream (an
    # event-record node costs a few us, so 7 steps in 8 carry none)
    t_start.record(env.stream)
    env.step_timed(args.steps)
    t_end.record(env.stream)
    t_end.synchronize()
    wall1 = time.time()
    barrier()
    ms = t_start.elapsed_time(t_end)
    s1 = env.stats()
    agent_steps = agent_steps_of(s1) - agent_steps_of(s0)
    births = sum(s["births"] for s in s1) - sum(s["births"] for s in s0)
    per_agent_bytes, n_alive_now = env.policy_bytes()
    per_agent_bytes = per_agent_bytes // max(1, n_alive_now)
    policy_bytes = agent_steps * per_agent_bytes
    region_ms, region_n, region_agents = env.policy_timing()

    # ---- policy-kernel timing pass: the same window after reset, every
    #      step's policy kernel between two CUDA events on the library stream
    #      (one-step graphs with event-record nodes), at least 10 launches;
    #      the roofline's source.  The timed region above times only the
    #      first step of each 8-step graph.
    env.reset()
    env.step(args.warmup)
    torch.cuda.synchronize()
    n_pass = max(args.steps, 10)
    env.step_timed(1)            # builds the one-step timed graph outside the pass
    env.policy_timing()
    env.reset()
    env.step(args.warmup)
    torch.cuda.synchronize()
    for _ in range(n_pass):
        env.step_timed(1)
    policy_ms, n_timed, timed_agents = env.policy_timing()

    # ---- end-to-end through the C-ABI: step + host read of the step's stats --
    env.reset()
    env.step(args.warmup)
    torch.cuda.synchronize()
    e0 = env.stats()
    barrier()
    # eco_step_read: each call enqueues a step and returns the records of the
    # step before it (their device -> host copy ends that step's graph), so
    # the host reads step s while step s + 1 runs; the last step's records
    # come from eco_read_stats, which synchronises
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tot, last = eco.eco_step_read(env.h, env.n_envs)
    tot, last = eco.eco_read_stats(env.h, env.n_envs)
    e_el = time.perf_counter() - t0
    barrier()
    wall2 = time.time()
    clk = clocks.stop(wall0, wall1, wall2) if clocks else None
    e_agent_steps = int(tot[:, 1].sum()) - agent_steps_of(e0)
    d2h = tot.nbytes + last.nbytes
    variant_name = eco.eco_policy_variant_name(env.variants()[1])
    sparse_forced = variant_name.startswith("input-sparse")
    launch_mode, launch_blocks = env.launch_mode()
    env.close()
    del env
    torch.cuda.empty_cache()

    # ---- batched only: the same worlds as separate handles, stepped one
    #      after another on one stream (64 sequential single-world launches)
    sequential = None
    if args.workload == "batched":
        shared = torch.cuda.Stream()
        singles = [eco.Env(e, stream=shared) for e in envs]
        for s in singles:
            s.reset()
            s.step(args.warmup)
        torch.cuda.synchronize()
        q0 = sum(agent_steps_of(s.stats()) for s in singles)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(shared)
        for _ in range(args.steps):
            for s in singles:
                eco.eco_step(s.h, 1)
        b.record(shared)
        b.synchronize()
        q1 = sum(agent_steps_of(s.stats()) for s in singles)
        qms = a.elapsed_time(b)
        sequential = {"value": (q1 - q0) / (qms * 1e-3), "unit": UNIT, "ms_per_step": qms / args.steps,
                      "how": "%d handles, one world each, eco_step(h, 1) in turn on one stream" % len(singles)}
        for s in singles:
            s.close()
        del singles
        torch.cuda.empty_cache()

    # ---- the input-sparse policy variants (opt-in: they stream only the
    #      W_in rows of nonzero inputs), same worlds and window; reported
    #      beside the dense figures, never as the roofline fraction
    sparse = None
    if args.workload != "batched" and args.policy_variant == 0:
        senv = eco.Env(envs, policy_variant=-1, launch_mode=args.launch_mode)
        senv.reset()
        senv.prepare()
        senv.step(args.warmup)
        torch.cuda.synchronize()
        q0 = agent_steps_of(senv.stats())
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(senv.stream)
        senv.step_timed(args.steps)
        b.record(senv.stream)
        b.synchronize()
        sms = a.elapsed_time(b)
        s_agent_steps = agent_steps_of(senv.stats()) - q0
        s_policy_ms, s_n, s_timed_agents = senv.policy_timing()
        sparse = {"value": s_agent_steps / (sms * 1e-3), "unit": UNIT,
                  "ms_per_step": sms / args.steps,
                  "policy_ms_per_step": s_policy_ms / max(1, s_n),
                  "effective_gbs": s_timed_agents * per_agent_bytes / (s_policy_ms * 1e-3) / 1e9
                  if s_policy_ms > 0 else None,
                  "variant": eco.eco_policy_variant_name(senv.variants()[1]),
                  "note": "streams only the W_in rows of nonzero inputs; effective_gbs = dense "
                          "algorithmic bytes / policy time (not a roofline fraction)"}
        senv.close()
        del senv
        torch.cuda.empty_cache()

    if dist is not None:
        ms, e_el, agent_steps, e_agent_steps = reduce_over_ranks(
            dist, [ms, e_el], [agent_steps, e_agent_steps], device="cuda")

    peaks, peak_kind = measured_peaks()
    # the timed launches' algorithmic bytes over their event-timed duration
    achieved = timed_agents * per_agent_bytes / (policy_ms * 1e-3) / 1e9 if policy_ms > 0 else 0.0
    region_achieved = region_agents * per_agent_bytes / (region_ms * 1e-3) / 1e9 if region_ms > 0 else None
    traffic = committed_traffic(w["name"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, _, _ = cpu_baseline_sample(w, args.cpu_seconds, (args.warmup, args.warmup + args.steps))
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": agent_steps / (ms * 1e-3),
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 (%s weights, int32 state)" % w["precision"],
            "data": "synthetic",
            "config": {
                "workload": ("batched: %d worlds (sides %s), %d slots, %d founders" % (
                    len(envs), "/".join(str(s) for s in sorted({e["side"] for e in envs})),
                    sum(e["slots"] for e in envs), sum(e["init_alive"] for e in envs)))
                if args.workload == "batched" else w["name"],
                "grid": "%dx%d" % (w["side"], w["side"]) if len(envs) == 1 else "mixed",
                "slots": sum(e["slots"] for e in envs),
                "founders": sum(e["init_alive"] for e in envs),
                "mlp": mlp_shape(w),
                "policy_form": w.get("policy_form", "plain"),
                "rules": w.get("rules", "simple"),
                "weights": w["precision"], "parallelism": "independent worlds, one per GPU",
                "l2": "inputs larger than L2 (%.2f GB of weights streamed per step)" %
                      (policy_bytes / max(1, args.steps) / 1e9),
                "window": "steps %d..%d after reset" % (args.warmup, args.warmup + args.steps),
                "mean_alive": agent_steps / max(1, args.steps) / world,
                "births": births,
                "policy_variant": variant_name,
                "env_phases": ("one persistent cooperative kernel, %d CTAs" % launch_blocks
                               if launch_mode == 0 else "one kernel per phase"),
            },
            "roofline": {
                "bound": "hbm", "kernel": "k_policy",
                # a forced input-sparse variant reads only some W_in rows, so
                # the dense byte count gives no roofline fraction for it
                "achieved": None if sparse_forced else achieved,
                "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": None if sparse_forced else achieved / float(peaks["hbm_gbs"]),
                "effective_gbs": achieved if sparse_forced else None,
                "peak_kind": "%s copy bandwidth" % peak_kind,
                "bytes_per_agent": per_agent_bytes,
                "policy_ms_per_step": policy_ms / max(1, n_timed),
                "policy_timing": "CUDA events around the policy kernel of every step of a timing "
                                 "pass over steps %d..%d after reset (one-step graphs; %d launches, "
                                 "%d agents)" % (args.warmup, args.warmup + n_pass, n_timed, timed_agents),
                "policy_timed_in_region": {
                    "launches": region_n, "agents": region_agents,
                    "achieved": None if sparse_forced else region_achieved,
                    "how": "CUDA events around the policy kernel of the first step of every 8-step "
                           "graph inside the timed region"},
                "policy_share_of_step": (policy_ms / max(1, n_timed)) / (ms / args.steps) if ms > 0 else None,
                "traffic": (traffic["dram_bytes_per_agent"] * agent_steps / max(1, args.steps * world))
                           if traffic and not sparse_forced else None,
                "traffic_source": traffic["source"] if traffic else None,
            },
            "e2e": {"value": e_agent_steps / e_el, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": kernels_per_step(launch_mode, w.get("rules", "simple")) * args.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if sequential is not None:
            line["sequential_single_world_launches"] = sequential
        if sparse is not None:
            line["input_sparse"] = sparse
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
