"""Benchmark: points/s of the full hull (filter + device hull) on one or more GB300s.

Default workload: the 1e8-point normal distribution (sigma 2^21, centred,
rounded and clamped to [0, 2^24)), inputs resident in HBM (800 MB, larger than
the 129 MB L2, so no flush is needed between steps).  One step = one ch_hull
call (all stages).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank runs an independent
replica of the workload (the single-hull path has no data-parallel exchange
on one GPU); value = all ranks' points / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Kernels per replayed hull: the filter part (init, sample, main, post) always;
# the large-survivor part (8 bucket kernels, the sort's histogram and 3 passes,
# which return at once on the bucketed path, and the chain merge) only when the
# post pass raised its graph condition.
FILTER_LAUNCHES = 4   # init, sample, main, post (the star pass adds one on large inputs)
LARGE_LAUNCHES = 13   # bk_prep, bk_hist, bk_bsum, bk_bstart, bk_items, bk_part1, bk_part2, bk_hull, sort_hist, 3 sort passes, chain
L2_BYTES = 129 * 1024 * 1024
HBM_NOMINAL_GBS = 7900.0   # GB300 HBM3e, nominal (context beside the measured copy bandwidth)
# One metric name for both arms (GPU library and the oracle's reference arm),
# so that their lines can be divided.
METRIC = "points/s (filter+hull, device-timed)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="normal_1e8")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--n", type=int, default=None, help="override the point count (testing)")
    ap.add_argument("--filter-steps", type=int, default=20,
                    help="timed ch_filter / ch_filter16 calls on the same input (0: skip)")
    ap.add_argument("--batched-sets", type=int, default=4096, help="sets of the batched workload (0: skip)")
    ap.add_argument("--batched-reps", type=int, default=5)
    ap.add_argument("--serve-requests", type=int, default=200000,
                    help="requests of the serving run, from the start of the 10 s stream (0: skip)")
    ap.add_argument("--serve-runs", type=int, default=3, help="repetitions of the serving run")
    ap.add_argument("--workloads", default="uniform_1e6,ring_1e8,distorted_1e8",
                    help="other single-hull workloads timed after the headline, comma-separated ('' to skip)")
    ap.add_argument("--workload-steps", type=int, default=30, help="timed steps of each extra workload")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(name, n):
    from synth import workloads as W
    kind, n0, seed = W.SINGLE[name]
    desc = {
        "normal": "isotropic normal, centre (2^23, 2^23), sigma 2^21, rounded, clamped to [0, 2^24)",
        "ring": "ring: angle U[0, 2pi), radius 2^23 - U[0, 64), rounded, clamped",
        "uniform": "uniform integers in [0, 2^24)^2",
        "distorted": "circumference with 2% distortion: angle U[0, 2pi), radius 2^23 (1 - 0.02 U[0, 1)), rounded, clamped",
    }[kind]
    return kind, (n or n0), seed, desc


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_from_profile(kernel, workload, n_bench):
    """Per-launch DRAM bytes of `kernel` from its committed ncu summary, scaled to
    the benchmark's point count; None when the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m_n = re.search(r"points_per_launch:\s*([0-9.eE+]+)", text)
    m_s = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    m_f = re.search(r"source_file:\s*(\S+)", text)
    if not (m_t and m_s and m_f):
        return None
    if source_sha(os.path.join(ROOT, m_f.group(1))) != m_s.group(1):
        return None
    scale = n_bench / float(m_n.group(1)) if m_n else 1.0
    return float(m_t.group(1)) * scale


def roofline_entry(kernel, algo_bytes, avg_launch_s, peak_gbs, peak_src, traffic):
    """The bench line's roofline object for an HBM-bound kernel: algorithmic
    bytes per launch over its average launch time, against the measured copy
    bandwidth (and, for context, the nominal HBM rate)."""
    achieved = algo_bytes / avg_launch_s / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
            "frac": achieved / peak_gbs, "peak_source": f"{peak_src} hbm_gbs",
            "frac_of_nominal": achieved / HBM_NOMINAL_GBS, "nominal_gbs": HBM_NOMINAL_GBS,
            "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": avg_launch_s * 1e3,
            "traffic": traffic}


def algorithmic_bytes(n, counters):
    """Algorithmic bytes per launch of each kernel of one hull with known byte
    counts, from the call's counters (raw survivors, records, mode): points
    are 8 bytes, a raw survivor 12 (its coordinates and index), a sort record
    12 (key and value).  Kernels whose time is latency (single blocks, merge
    tree) have no entry."""
    raw, m, two_pass = counters["raw"], counters["records"], counters["two_pass"]
    out = {"main_filter": 8.0 * n + 12.0 * raw,
           "post": (8.0 * n if two_pass else 12.0 * raw) + 12.0 * m}
    if counters["stage"] >= 1:
        out.update({"bk_hist": 4.0 * m, "bk_part1": 24.0 * m, "bk_part2": 24.0 * m, "bk_hull": 12.0 * m})
    return out


def kernel_rooflines(prof, algo, peak, peak_src, workload, n):
    """Per-kernel achieved GB/s for the kernels with algorithmic bytes, and the
    roofline object of the one with the largest device time among them."""
    per = {}
    for k, b in algo.items():
        if k in prof and prof[k][0]:
            avg_s = prof[k][1] / prof[k][0] / 1e3
            per[k] = {"avg_ms": avg_s * 1e3, "algorithmic_bytes": b, "achieved_gbs": b / avg_s / 1e9,
                      "frac_of_measured_hbm": b / avg_s / 1e9 / peak}
    if not per:
        return per, None
    top = max(per, key=lambda k: per[k]["avg_ms"])
    roof = roofline_entry(top, algo[top], per[top]["avg_ms"] / 1e3, peak, peak_src,
                          traffic_from_profile(top, workload, n))
    return per, roof


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(kind, seed, seconds):
    """The oracle as it stands, single-threaded, on a bounded sample of the workload."""
    import oracle
    from synth import workloads as W
    n = 2_000_000
    pts = W.make(kind, n, seed)
    oracle.hull(pts[:1000])
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.hull(pts)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": n * reps / el, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x {n} points of the same {kind} distribution (seed {seed}), "
                      f"single-threaded C Andrew monotone chain, {el:.1f} s"}


def cpu_heaphull(kind, seed, seconds):
    """The CPU heaphull comparator (oracle/heaphull_cpu.c: parallel extremes and
    octagon filter, parallel sort, Andrew's chains) on one thread and on every
    host core, on the same bounded sample as the CPU baseline."""
    import oracle
    from synth import workloads as W
    n = 2_000_000
    pts = W.make(kind, n, seed)
    cores = os.cpu_count() or 1
    out = {"unit": "points/s", "cores": cores, "kind": "CPU heaphull (POSIX threads)"}
    for label, threads in (("value_1_thread", 1), ("value_all_cores", cores)):
        oracle.heaphull_cpu(pts[:1000], threads)
        reps, t0 = 0, time.perf_counter()
        while True:
            oracle.heaphull_cpu(pts, threads)
            reps += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
        out[label] = n * reps / el
    out["sample"] = f"{n} points of the same {kind} distribution (seed {seed}), about {seconds:.1f} s per setting"
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    kind, n, seed, desc = workload_config(args.workload, args.n)
    import oracle
    from synth import workloads as W
    # per-step sample sized so the whole run stays near 90 s of single-core work
    # (the oracle runs ~8e6 points/s on one core)
    sample = int(min(1_000_000, max(10_000, 90.0 * 8e6 / max(1, args.steps + args.warmup))))
    pts = W.make(kind, sample, seed)
    for _ in range(args.warmup):
        oracle.hull(pts)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.hull(pts)
    el = time.perf_counter() - t0
    value = sample * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "distribution": desc,
                   "reference_step": f"oracle on a {sample}-point sample of the workload"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample} points of the same {kind} distribution per step"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    # the rank's device first: the process group's barriers and reductions
    # then run on it rather than on device 0
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from __graft_entry__ import build
    build()
    import paper_2209_12310_gb300 as ch
    from synth import workloads as W

    kind, n, seed, desc = workload_config(args.workload, args.n)
    host = W.make(kind, n, seed)
    pts = torch.from_numpy(host).cuda()
    out_idx = torch.empty(n, dtype=torch.int32, device="cuda")
    out_n = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def step():
        ch.ch_hull(pts.data_ptr(), n, out_idx.data_ptr(), out_n.data_ptr(), sp)

    ch.ch_reserve(n, 1, sp)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    h = int(out_n.item())
    if h < 0:
        raise SystemExit(f"hull failed: {ch.ch_strerror(h)}")

    def barrier():
        if world > 1:
            dist.barrier()

    # Timed region: device events around exactly K steps (repeated calls replay
    # the library's cached CUDA graph of the launch sequence).
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    in_l2 = 8 * n <= L2_BYTES
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda") if in_l2 else None
    barrier()
    torch.cuda.synchronize()
    if not in_l2:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    else:
        # inputs fit in L2: each step timed alone, L2 overwritten in between
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a, b in evs:
            flush_buf.fill_(1)
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
    barrier()
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n * args.steps / (ms / 1e3)

    # Per-kernel device times: the library records CUDA events around each
    # kernel on the launching stream (direct launches while enabled), over a
    # second region of the same workload.
    prof_steps = min(args.steps, 200)
    ch.ch_profile_reset()
    ch.ch_profile_enable(True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    ch.ch_profile_enable(False)
    prof = ch.ch_profile_read()

    # Roofline of the dominant kernel (largest device time among the kernels
    # with algorithmic byte counts) and of the whole step.
    peak, peak_src = peaks()
    counters = ch.ch_hull_counters(sp)
    algo = algorithmic_bytes(n, counters)
    per_kernel, roof = kernel_rooflines(prof, algo, peak, peak_src, args.workload, n)
    kernels = {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in prof.items()}
    kernels["_region"] = f"{prof_steps} profiled steps after the timed region"
    for k, v in per_kernel.items():
        kernels[k].update({kk: v[kk] for kk in ("algorithmic_bytes", "achieved_gbs", "frac_of_measured_hbm")})
    # Kernels of a replayed step: the filter part, the star pass on its side
    # branch when the input has enough tiles for it, and the large-survivor
    # part when the call's counters say it ran (its graph node is skipped
    # otherwise).
    large = counters.get("stage", 0) >= 1
    launches_per_step = FILTER_LAUNCHES + (1 if "star" in prof else 0) + (LARGE_LAUNCHES if large else 0)

    step_bytes = sum(v["algorithmic_bytes"] for v in per_kernel.values())
    step_roof = {"algorithmic_bytes": step_bytes, "achieved_gbs": step_bytes / (ms / args.steps / 1e3) / 1e9,
                 "frac_of_measured_hbm": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
                 "note": "every kernel's algorithmic bytes over the whole step time"}
    # The serving leg replays a 10 s stream in real time; it runs before the
    # legs that leave large workspaces behind (the 1e8-point workloads, the
    # 4096-set batch): measured after them, its p99 rose from about 10 ms to
    # 35-410 ms (the cause is not the Python garbage collector).
    serving = run_serving(ch, torch, args) if (args.serve_requests > 0 and world == 1) else None
    filters = run_filters(ch, torch, args, pts, n, sp, peak) if (args.filter_steps > 0 and world == 1) else None
    others = [w for w in args.workloads.split(",") if w and w != args.workload]
    workloads = run_workloads(ch, torch, args, others, sp, peak, peak_src, local) \
        if (others and world == 1) else None
    batched = run_batched(ch, torch, args, sp) if (args.batched_sets > 0 and world == 1) else None

    # End to end through the host-buffer entry point: pinned input, H2D, hull, D2H.
    import ctypes
    pinned = torch.from_numpy(host).pin_memory()
    out_host = torch.empty(n, dtype=torch.int32).pin_memory()
    hn = ctypes.c_int64()
    ch.ch_hull_host(pinned.data_ptr(), n, out_host.data_ptr(), ctypes.addressof(hn), sp)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ch.ch_hull_host(pinned.data_ptr(), n, out_host.data_ptr(), ctypes.addressof(hn), sp)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * n * args.e2e_steps / e2e_s, "unit": "points/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 + 4 * int(hn.value),
           "steps": args.e2e_steps, "entry_point": "ch_hull_host (pinned host buffers)"}

    if rank == 0:
        cpu = cpu_baseline(kind, seed, args.cpu_seconds) if world == 1 else None
        if cpu is not None:   # the multi-core comparator, part of the same CPU-baseline leg
            cpu["heaphull_comparator"] = cpu_heaphull(kind, seed, max(0.5, args.cpu_seconds / 4))
        line = {
            "metric": METRIC, "value": value, "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "distribution": desc, "seed": seed,
                       "hull_vertices": h,
                       "l2": (f"inputs {8 * n / 1e6:.0f} MB per step, below the 129 MB L2: L2 overwritten "
                              "(256 MB write) before each step, steps timed one by one") if in_l2 else
                             f"inputs {8 * n / 1e6:.0f} MB per step > 129 MB L2 (no flush needed)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "step_roofline": step_roof, "counters": counters, "kernels": kernels,
            "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": launches_per_step * args.steps, "clocks": clk,
        }
        if filters is not None:
            line["filters"] = filters
        if workloads is not None:
            line["workloads"] = workloads
        if batched is not None:
            line["batched"] = batched
        if serving is not None:
            line["serving"] = serving
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_workloads(ch, torch, args, names, sp, peak, peak_src, gpu_index):
    """The other single-hull workloads, each timed like the headline (device
    events around K steps on the resident input; L2 overwritten before each
    step when the input fits in it), with per-kernel device times, the
    roofline of its dominant kernel and the step's fraction of HBM."""
    from synth import workloads as W
    out = {}
    for name in names:
        kind, n, seed, desc = workload_config(name, None)
        host = W.make(kind, n, seed)
        pts = torch.from_numpy(host).cuda()
        out_idx = torch.empty(n, dtype=torch.int32, device="cuda")
        out_n = torch.empty(1, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()

        def step():
            ch.ch_hull(pts.data_ptr(), n, out_idx.data_ptr(), out_n.data_ptr(), sp)

        ch.ch_reserve(n, 1, sp)
        for _ in range(5):
            step()
        torch.cuda.synchronize()
        h = int(out_n.item())
        if h < 0:
            raise SystemExit(f"{name}: hull failed: {ch.ch_strerror(h)}")
        K = max(3, args.workload_steps)
        in_l2 = 8 * n <= L2_BYTES
        flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda") if in_l2 else None
        clocks = ClockSampler(gpu_index)
        clocks.start()
        time.sleep(0.2)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K if in_l2 else 1)]
        if in_l2:
            for a, b in evs:
                flush_buf.fill_(1)
                a.record(stream)
                step()
                b.record(stream)
        else:
            evs[0][0].record(stream)
            for _ in range(K):
                step()
            evs[0][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in evs) / K
        ch.ch_profile_reset()
        ch.ch_profile_enable(True)
        for _ in range(min(K, 10)):
            if in_l2:
                flush_buf.fill_(1)
            step()
        torch.cuda.synchronize()
        ch.ch_profile_enable(False)
        prof = ch.ch_profile_read()
        counters = ch.ch_hull_counters(sp)
        algo = algorithmic_bytes(n, counters)
        per_kernel, roof = kernel_rooflines(prof, algo, peak, peak_src, name, n)
        kernels = {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in prof.items()}
        for k, v in per_kernel.items():
            kernels[k].update({kk: v[kk] for kk in ("algorithmic_bytes", "achieved_gbs", "frac_of_measured_hbm")})
        step_bytes = sum(v["algorithmic_bytes"] for v in per_kernel.values())
        out[name] = {
            "n": n, "distribution": desc, "seed": seed, "hull_vertices": h, "steps": K,
            "ms_per_step": ms, "points_per_s": n / (ms / 1e3),
            "l2": "L2 overwritten (256 MB write) before each step, steps timed one by one" if in_l2 else
                  f"inputs {8 * n / 1e6:.0f} MB > 129 MB L2 (no flush needed)",
            "counters": counters, "roofline": roof,
            "step_roofline": {"algorithmic_bytes": step_bytes,
                              "achieved_gbs": step_bytes / (ms / 1e3) / 1e9,
                              "frac_of_measured_hbm": step_bytes / (ms / 1e3) / 1e9 / peak},
            "kernels": kernels, "clocks": clk,
        }
        del pts, out_idx, out_n, flush_buf
        torch.cuda.empty_cache()
    return out


def run_filters(ch, torch, args, pts, n, sp, peak):
    """The filter on its own (labels and queue sizes) with the octagon
    (ch_filter) and with the 16-direction polygon (ch_filter16), on the
    resident input: device time per call, points kept, and the HBM fraction
    of each pass (8 bytes a point read; the label pass also writes 1)."""
    labels = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    counts = torch.empty(4, dtype=torch.int64, device="cuda")
    ext = torch.empty(16, dtype=torch.int32, device="cuda")
    out = {}
    for name, fn, passes in (("octagon", ch.ch_filter, {"main_filter": 8.0, "labels": 9.0}),
                             ("octagon, two-kernel Manhattan extremes", ch.ch_filter_manhattan,
                              {"manhattan_axis": 8.0, "manhattan_corner": 8.0, "labels": 9.0}),
                             ("16-gon", ch.ch_filter16, {"filter16_extremes": 8.0, "filter16_labels": 9.0})):
        def call():
            fn(pts.data_ptr(), n, ext.data_ptr(), labels.data_ptr(), counts.data_ptr(), sp)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.filter_steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.filter_steps
        ch.ch_profile_reset()
        ch.ch_profile_enable(True)
        for _ in range(args.filter_steps):
            call()
        torch.cuda.synchronize()
        ch.ch_profile_enable(False)
        prof = ch.ch_profile_read()
        kept = int(counts.sum().item())
        per = {}
        for k, bpp in passes.items():
            if k in prof and prof[k][0]:
                avg_ms = prof[k][1] / prof[k][0]
                gbs = bpp * n / (avg_ms / 1e3) / 1e9
                per[k] = {"avg_ms": avg_ms, "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak}
        out[name] = {"ms_per_call": ms, "points_per_s": n / (ms / 1e3), "kept": kept,
                     "kept_fraction": kept / max(n, 1), "passes": per}
    out["note"] = ("labels + queue sizes of every point; octagon = ch_filter (extremes fused in one pass), "
                   "two-kernel Manhattan = ch_filter_manhattan (the paper's Sec. 3 form: axis extremes, then "
                   "minimum Manhattan distance to the box corners), 16-gon = ch_filter16 "
                   f"(same input, {args.filter_steps} calls each, CUDA events)")
    return out


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def run_batched(ch, torch, args, sp):
    """4096 sets of log-uniform size in [100, 1e6] (uniform/normal/ring) in one
    ch_hull_batched call, against one ch_hull call per set on the same GPU."""
    from synth import workloads as W
    k = args.batched_sets
    pts_h, off_h = W.batched(k)
    total = int(off_h[-1])
    d = torch.from_numpy(pts_h).cuda()
    doff = torch.from_numpy(off_h).cuda()
    out_idx = torch.empty(total, dtype=torch.int32, device="cuda")
    out_n = torch.empty(k, dtype=torch.int64, device="cuda")
    lib = ch.load()

    def batch():
        st = lib.ch_hull_batched(d.data_ptr(), doff.data_ptr(), k, out_idx.data_ptr(), out_n.data_ptr(),
                                 off_h.ctypes.data, sp)
        if st != 0:
            raise SystemExit(f"ch_hull_batched failed: {ch.ch_strerror(st)}")

    t0 = time.perf_counter()
    batch()   # the first batch of this size class also runs the tile-shape autotuner
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    batch()
    torch.cuda.synchronize()
    lat = []
    for _ in range(args.batched_reps):
        t0 = time.perf_counter()
        batch()
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0) * 1e3)
    # per-kernel device times of the batch (direct launches while profiling)
    ch.ch_profile_reset()
    ch.ch_profile_enable(True)
    for _ in range(3):
        batch()
    torch.cuda.synchronize()
    ch.ch_profile_enable(False)
    prof = ch.ch_profile_read()
    peak, _ = peaks()
    filt = {}
    for kname in ("batched_extremes", "batched_filter"):   # each streams every point once
        if kname in prof and prof[kname][0]:
            avg_s = prof[kname][1] / prof[kname][0] / 1e3
            filt[kname] = {"avg_ms": avg_s * 1e3, "algorithmic_bytes": 8.0 * total,
                           "achieved_gbs": 8.0 * total / avg_s / 1e9,
                           "frac_of_measured_hbm": 8.0 * total / avg_s / 1e9 / peak}
    if len(filt) == 2:
        both_s = sum(v["avg_ms"] for v in filt.values()) / 1e3
        filt["filter_total"] = {"algorithmic_bytes": 8.0 * total, "avg_ms": both_s * 1e3,
                                "frac_of_measured_hbm": 8.0 * total / both_s / 1e9 / peak,
                                "note": "one 8-byte read of every point is the filter's algorithmic traffic"}
    kernels = {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in prof.items()}
    ref_idx = torch.empty_like(out_idx)
    ref_n = torch.empty_like(out_n)

    def one_per_launch():
        for i in range(k):
            lib.ch_hull(d[int(off_h[i]):].data_ptr(), int(off_h[i + 1] - off_h[i]), ref_idx[int(off_h[i]):].data_ptr(),
                        ref_n[i:].data_ptr(), sp)

    one_per_launch()
    torch.cuda.synchronize()
    lat1 = []
    for _ in range(2):
        t0 = time.perf_counter()
        one_per_launch()
        torch.cuda.synchronize()
        lat1.append((time.perf_counter() - t0) * 1e3)
    same = bool(torch.equal(ref_n, out_n))
    if same:
        ns = out_n.cpu().numpy()
        mask = torch.zeros(total, dtype=torch.bool, device="cuda")
        for i in range(k):
            mask[int(off_h[i]):int(off_h[i]) + int(ns[i])] = True
        same = bool(torch.equal(out_idx[mask], ref_idx[mask]))
    p50 = _pct(lat, 50)
    return {"workload": f"{k} sets, sizes log-uniform [100, 1e6], uniform/normal/ring, seed 3",
            "points": total, "batches": len(lat), "latency_ms_p50": p50, "latency_ms_p99": _pct(lat, 99),
            "points_per_s": total / (p50 / 1e3),
            "one_per_launch": {"latency_ms_p50": _pct(lat1, 50), "points_per_s": total / (_pct(lat1, 50) / 1e3),
                               "calls_per_batch": k},
            "same_result_as_one_per_launch": same,
            "filter_hbm": filt, "kernels": kernels,
            "tile_shape": dict(zip(("threads", "points_per_thread"), ch.ch_batched_config(total, k))),
            "first_call_ms_with_tuning": first_ms,
            "timing": "host clock around each call plus a device synchronize (the call itself reads a small "
                      "device array of per-set flags)"}


def batch_trace_summary(trace):
    """Per-batch server trace (ch_server_trace) in a few numbers: p50 / p99 of
    the batch size and of each phase, and the mean phases of the slowest 1 %
    of the batches (by host time from formation to retirement)."""
    if not trace:
        return None
    import numpy as np
    t = np.array(trace, dtype=np.float64)
    cols = {"requests": 1, "points": 2, "copy_in_ms": 3, "hull_ms": 4, "copy_out_ms": 5, "host_ms": 6}
    out = {"batches": int(t.shape[0]), "sets_redone": int(t[:, 7].sum())}
    for name, c in cols.items():
        out[name + "_p50"] = float(np.percentile(t[:, c], 50))
        out[name + "_p99"] = float(np.percentile(t[:, c], 99))
    slow = t[t[:, 6] >= np.percentile(t[:, 6], 99)]
    out["slowest_1pct_mean"] = {name: float(slow[:, c].mean()) for name, c in cols.items()}
    out["slowest_1pct_mean"]["sets_redone"] = float(slow[:, 7].mean())
    return out


def run_serving(ch, torch, args):
    """Poisson request stream (20,000/s, sizes log-uniform [1e3, 1e7], 50% normal /
    40% uniform / 10% ring) replayed for its first R requests into the
    continuous-batching server (16 GB budget), args.serve_runs times; then the
    plain path: the first 4000 requests served one ch_hull_host call after
    another by one thread, each started no earlier than its arrival time
    (a measured FIFO server, not a model)."""
    import ctypes

    import numpy as np
    from synth import workloads as W
    arrivals, sizes, names = W.serving_plan()
    R = min(args.serve_requests, len(arrivals))
    arrivals, sizes, names = arrivals[:R], sizes[:R], names[:R]
    # a pool of pre-generated requests covering the size range (pinned host
    # memory); request i uses the pool entry of its kind nearest in log size
    pool = {}
    grid = np.exp(np.linspace(np.log(1e3), np.log(1e7), 24))
    for kind in ("normal", "uniform", "ring"):
        ents = []
        for j, sz in enumerate(grid):
            arr = torch.from_numpy(np.ascontiguousarray(W.make(kind, int(sz), 500 + j))).pin_memory()
            ents.append((int(sz), arr))
        pool[kind] = ents
    reqs = []
    for i in range(R):
        ents = pool[str(names[i])]
        j = int(np.argmin([abs(np.log(e[0]) - np.log(sizes[i])) for e in ents]))
        reqs.append(ents[j])
    pts_total = sum(r[0] for r in reqs)
    lib = ch.load()

    # (no nvidia-smi sampling here: its queries stall the server's CUDA calls,
    # measured at p50 3 ms without against 10-25 ms with a 50 ms sampler)
    def serve_once():
        srv = ch.ch_server_create(16 << 30, torch.cuda.current_device())
        try:
            t0 = time.perf_counter()
            i = 0
            outstanding = []
            bufs = {}
            while i < R or outstanding:
                now = time.perf_counter() - t0
                while i < R and arrivals[i] <= now:
                    st, t = ch.ch_submit(srv, reqs[i][1].data_ptr(), reqs[i][0])
                    if st == ch.CH_EBUSY:
                        break
                    if st != 0:
                        raise SystemExit(f"ch_submit failed: {ch.ch_strerror(st)}")
                    outstanding.append((t, reqs[i][0]))
                    i += 1
                keep = []
                for t, nn in outstanding[:64]:   # completions are nearly FIFO
                    buf = bufs.setdefault(nn, np.empty(nn, np.int32))
                    st, h = ch.ch_poll(srv, t, buf.ctypes.data, nn)
                    if st == ch.CH_PENDING:
                        keep.append((t, nn))
                    elif st != 0:
                        raise SystemExit(f"ch_poll failed: {ch.ch_strerror(st)}")
                outstanding = keep + outstanding[64:]
                if time.perf_counter() - t0 > 120:
                    break
                time.sleep(0.0002)
            wall = time.perf_counter() - t0
            stats = ch.ch_server_stats(srv)
            trace = ch.ch_server_trace(srv)
        finally:
            ch.ch_server_destroy(srv)
        return {"completed": stats["completed"], "wall_s": wall, "latency_ms_p50": stats["p50_ms"],
                "latency_ms_p99": stats["p99_ms"], "points_per_s": pts_total / wall,
                "batches": batch_trace_summary(trace)}

    # the arrival loop runs in Python: a garbage-collector pass in the middle
    # of it would hold back the submissions behind it (a burst afterwards),
    # so the collector is off while the streams are replayed
    import gc
    gc.collect()
    gc.disable()
    try:
        runs = [serve_once() for _ in range(max(1, args.serve_runs))]
    finally:
        gc.enable()

    # the plain path, measured: one thread, one blocking ch_hull_host per
    # request in arrival order, each started no earlier than its arrival
    m = min(4000, R)
    out = np.empty(int(max(r[0] for r in reqs[:m])), np.int32)
    hn = ctypes.c_int64()
    lib.ch_hull_host(reqs[0][1].data_ptr(), reqs[0][0], out.ctypes.data, ctypes.addressof(hn), 0)
    lat1 = []
    t0 = time.perf_counter()
    for j in range(m):
        while time.perf_counter() - t0 < arrivals[j]:
            time.sleep(0.00005)
        lib.ch_hull_host(reqs[j][1].data_ptr(), reqs[j][0], out.ctypes.data, ctypes.addressof(hn), 0)
        lat1.append((time.perf_counter() - t0 - arrivals[j]) * 1e3)
    wall1 = time.perf_counter() - t0
    pts_m = sum(r[0] for r in reqs[:m])
    p50s = [r["latency_ms_p50"] for r in runs]
    p99s = [r["latency_ms_p99"] for r in runs]
    rates = [r["points_per_s"] for r in runs]
    return {"workload": f"first {R} requests of the 10 s Poisson stream at 20,000/s (sizes log-uniform [1e3, 1e7], "
                        "50% normal / 40% uniform / 10% ring, seed 4), pooled pre-generated pinned inputs",
            "requests": R, "points": pts_total, "runs": runs, "budget_bytes": 16 << 30,
            "completed": runs[len(runs) // 2]["completed"],
            "latency_ms_p50": statistics.median(p50s), "latency_ms_p99": statistics.median(p99s),
            "latency_ms_p50_range": [min(p50s), max(p50s)], "latency_ms_p99_range": [min(p99s), max(p99s)],
            "points_per_s": statistics.median(rates),
            "one_per_launch": {"requests": m, "latency_ms_p50": _pct(lat1, 50), "latency_ms_p99": _pct(lat1, 99),
                               "points_per_s": pts_m / wall1, "wall_s": wall1,
                               "entry_point": "ch_hull_host per request, one thread, each request started no "
                                              "earlier than its arrival (measured)"}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
