"""Benchmark: rays/s to z = 1 through an AMR potential on one GB300 (or N replicas).

Workload (synthetic, seeded): 256^3 coarse grid in a 1 h^-1 Gpc box plus 3 refinement
levels (2%, 0.5%, 0.125% of the volume) on the densest cells, FP32 phi/grad phi records,
two time slices (z = 0, 1) linear in eta, 786,432 HEALPix (nside 256, NESTED) rays from
the box centre to z = 1, 4 RK4 steps per AMR cell, FP64 ray state.

One timed step = one mt_trace_rays call over all rays (the whole hot path: locate, CIC
with level fallback, geodesic RHS, RK4, stop, outputs).  The field (1.2 GB) is larger
than L2, and L2 is also flushed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reported CPU baseline) on a bounded
sample of the same rays on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RK4 geodesic steps/s and rays/s to z=1 on AMR field; % of HBM roofline"
UNIT = "rays/s"
FIELD_BYTES_PER_STEP = 4 * 8 * 16 * 2   # 4 stages x 8 CIC records x 16 B (float4) x 2 bracketing slices
# the same per interpolation scheme: NGP reads 1 cell per stage, CIC 8, TSC 27 (Eqs. 7-9)
FIELD_BYTES_BY_SCHEME = {"ngp": 4 * 1 * 16 * 2, "cic": FIELD_BYTES_PER_STEP, "tsc": 4 * 27 * 16 * 2}


# ncu record of trace_kernel<float> on the benchmark workload, with the SHA-256 of the kernel's code
# (its sources with comments removed) at capture time; reported only while that code is unchanged.
# Every figure comes from single-pass captures of full benchmark launches (1,907,632,740 RK4 steps),
# one metric per capture:
#   dram_bytes_per_launch: dram__bytes_read.sum + dram__bytes_write.sum;
#   per_rk4_step: warp_inst = smsp__inst_executed.sum / steps; fp64_lane_slots = FP64-pipe lane slots
#       occupied per step = sm__pipe_fp64_cycles_active.sum x 2 lanes per cycle (the pipe's peak, 2
#       DFMA lanes per cycle per SM; a warp instruction holds it 16 cycles) / steps;
#   pct: fp64_pipe = sm__pipe_fp64_cycles_active.sum / sm__cycles_active.sum; issue_active =
#       smsp__inst_executed.sum / (4 x sm__cycles_active.sum) (instructions per scheduler cycle);
#       lanes_per_inst = smsp__thread_inst_executed.sum / smsp__inst_executed.sum; dram_throughput =
#       the DRAM bytes over the launch time against the measured copy rate.
TRACE_KERNEL_SOURCES = ["include/mt.h", "paper_2111_08744_gb300/csrc/mt_internal.cuh",
                        "paper_2111_08744_gb300/csrc/mt_mixed.cuh", "paper_2111_08744_gb300/csrc/mt_trace_device.cuh",
                        "paper_2111_08744_gb300/csrc/mt_trace.cu"]
NCU_RECORD = {"sources_sha256": "2368f9aab23d743202379115c02b85402050b066535b7419fec988e027c320c6",
              "dram_bytes_per_launch": 57878603008 + 993063680,
              "per_rk4_step": {"warp_inst": 111.280, "fp64_lane_slots": 65.335},
              "pct": {"fp64_pipe": 55.80, "issue_active": 47.52, "lanes_per_inst": 19.18, "dram_throughput": 2.45}}
SMS, SCHEDULERS_PER_SM = 152, 4


def _strip_comments(text: str) -> str:
    """C/C++ source without // and /* */ comments (string and character literals kept), with every
    run of white space reduced to one blank."""
    import re
    pat = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'', re.S)
    code = pat.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", text)
    return " ".join(code.split())


def trace_kernel_sha256():
    """SHA-256 of the trace kernel's code: its sources with the comments removed, so that a change
    of comments keeps the ncu record and a change of code drops it."""
    import hashlib
    h = hashlib.sha256()
    for rel in TRACE_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel)) as f:
            h.update(rel.encode() + b"\0" + _strip_comments(f.read()).encode())
    return h.hexdigest()


def ncu_record():
    """The ncu record of the trace kernel, or None once the kernel's code changed since the capture."""
    if NCU_RECORD["sources_sha256"] and NCU_RECORD["sources_sha256"] == trace_kernel_sha256():
        return NCU_RECORD
    return None


def measured_traffic():
    """ncu DRAM bytes of one trace launch, or None once the kernel changed since the capture."""
    rec = ncu_record()
    return rec["dram_bytes_per_launch"] if rec else None


def roofline(total_steps, ms, sm_mhz, fp64_fma_per_s, hbm_gbs, field_bytes, record, peaks_source,
             missing="stale: the trace kernel changed since the last ncu capture"):
    """Roofline of the trace kernel.  The binding resource is arithmetic issue, not HBM (the field
    gathers are served by shared memory, L1 and L2): the headline is the FP64 pipe -- the FP64 lane
    slots it occupies per RK4 step (ncu) x RK4 steps per second (CUDA events), against the FP64 FMA
    lane rate measured on this GPU by mt_probe_fp64_fma_rate -- with the issue-slot fraction, the
    DRAM fraction (ncu traffic) and the algorithmic field bandwidth ("effective") beside it."""
    t = ms * 1e-3
    steps_per_s = total_steps / t
    eff = field_bytes * steps_per_s / 1e9
    out = {"bound": "alu", "unit": "G FP64 lane-slots/s", "achieved": None, "peak": fp64_fma_per_s / 1e9,
           "frac": None, "traffic": None, "kernel": "trace_kernel<float>",
           "peak_source": "mt_probe_fp64_fma_rate, measured in this run (of measured)",
           "limiter": "latency-bound issue: FP64 pipe and issue slots share the time, DRAM is not the limit",
           "hbm_effective": {"algorithmic_bytes_per_rk4_step": field_bytes, "achieved_GBs": eff, "peak_GBs": hbm_gbs,
                             "frac": eff / hbm_gbs, "peak_source": peaks_source},
           "rk4_steps_per_launch": total_steps}
    if record is None:
        out["ncu_record"] = missing
        return out
    per = record["per_rk4_step"]
    if per.get("fp64_lane_slots"):
        ach = per["fp64_lane_slots"] * steps_per_s
        out["achieved"] = ach / 1e9
        out["frac"] = ach / fp64_fma_per_s
    if per.get("warp_inst") and sm_mhz:
        issue_peak = SMS * SCHEDULERS_PER_SM * sm_mhz * 1e6
        out["issue"] = {"achieved_ginst_s": per["warp_inst"] * steps_per_s / 1e9, "peak_ginst_s": issue_peak / 1e9,
                        "frac": per["warp_inst"] * steps_per_s / issue_peak}
    if record.get("dram_bytes_per_launch"):
        out["traffic"] = record["dram_bytes_per_launch"]
        dram = record["dram_bytes_per_launch"] / t / 1e9
        out["dram"] = {"achieved_GBs": dram, "peak_GBs": hbm_gbs, "frac": dram / hbm_gbs}
    out["ncu_pct"] = record.get("pct", {})
    return out


def workload_config(w):
    cells = [int(l.keys.size) for l in w.levels]
    return {"workload": "AMR 256^3 + 3 levels, 786,432 rays to z=1 (mixed: FP32 field, FP64 state)",
            "box_h-1Mpc": w.box, "n_coarse": w.n_coarse, "n_levels": w.n_levels, "cells_per_level": cells,
            "n_slices": w.n_slices, "n_rays": w.n_rays, "z_max": float(w.z_max[0]),
            "steps_per_cell": w.steps_per_cell, "field_precision": "fp32", "state_precision": "fp64",
            "l2": "field 1.2 GB > L2; L2 flushed between timed steps"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(w, rank, ws):
    """Weak scaling: each rank traces its own light cone (same field, same rays) from an
    observer shifted by rank/ws of the box along x; no data moves between ranks."""
    if ws == 1:
        return w
    import dataclasses
    obs = w.observer.copy()
    obs[:, 0] = (obs[:, 0] + w.box * rank / ws) % w.box
    return dataclasses.replace(w, observer=obs)


def oracle_sample(w, budget_s=15.0, interp="cic"):
    """Time the CPU oracle on a bounded, seeded sample of the rays; returns (rays/s, n, threads, secs)."""
    import oracle
    threads = oracle.default_threads()
    rng = np.random.Generator(np.random.PCG64(2024))
    n = 64
    while True:
        idx = np.sort(rng.choice(w.n_rays, size=n, replace=False))
        t0 = time.perf_counter()
        oracle.trace(w, dirs=w.dirs[:, idx], n_threads=threads, interp=interp)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or n >= w.n_rays:
            return n / dt, n, threads, dt
        n = min(w.n_rays, int(n * min(8.0, max(2.0, budget_s / max(dt, 1e-3) / 2))))


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2111_08744_gb300 import inputs as I
    w = I.cached(I.config_amr)
    vals = []
    for i in range(args.warmup + args.steps):
        v, n, threads, dt = oracle_sample(w, budget_s=args.ref_budget, interp=args.interp)
        if i >= args.warmup:
            vals.append((v, n, dt))
    value = float(np.mean([v for v, _, _ in vals]))
    n = vals[-1][1]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean([d for _, _, d in vals]) * 1e3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w), interp=args.interp),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.default_threads(),
                             "kind": "oracle", "sample": f"{n} seeded rays of the 786,432 per step, FP64 field"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank):
    import torch

    from paper_2111_08744_gb300 import binding as B
    from paper_2111_08744_gb300 import build as Bd
    from paper_2111_08744_gb300 import inputs as I

    Bd.build()
    w = rank_workload(I.cached(I.config_amr), rank, ws)
    if args.rays:
        # a seeded subset of the rays (profiling captures of a short launch; not a bench line)
        rng = np.random.Generator(np.random.PCG64(7))
        w = I.with_rays(w, w.dirs[:, np.sort(rng.choice(w.n_rays, size=args.rays, replace=False))])
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    levels32 = I.fp32_levels(w)
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, levels32, w.bg, "fp32")
    params = B.TraceParams.from_workload(w, interp=args.interp)
    n = w.n_rays
    dirs = torch.from_numpy(w.dirs).to(dev)
    out = B.alloc_outputs(n, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        B.trace_rays(tree, params, dirs, out)
    torch.cuda.synchronize()
    st = tree.device_status()
    if st != B.MT_OK:
        raise RuntimeError(f"device status after warm-up: {B.status_str(st)}")
    total_steps = int(out["n_steps"].sum().item())

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        B.trace_rays(tree, params, dirs, out)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(times))
    ms_max = max_over_ranks(ms, ws)
    if int(out["n_steps"].sum().item()) != total_steps:
        raise RuntimeError("step count changed between launches")
    value = ws * n / (ms_max * 1e-3)
    steps_per_s = ws * total_steps / (ms_max * 1e-3)

    # end to end through the public API: host (pinned) directions in, host outputs back
    host_dirs = torch.from_numpy(w.dirs).pin_memory()
    host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    h2d = host_dirs.numel() * 8
    d2h = sum(v.numel() * v.element_size() for v in out.values())
    e2e_ms = []
    for i in range(max(1, min(args.steps, 3)) + 1):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        d = host_dirs.to(dev, non_blocking=True)
        B.trace_rays(tree, params, d, out)
        for k in out:
            host_out[k].copy_(out[k], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            e2e_ms.append(a.elapsed_time(b))
    e2e_value = ws * n / (max_over_ranks(float(np.mean(e2e_ms)), ws) * 1e-3)

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_rate = B.probe_fp64_fma_rate()
    record = ncu_record() if (args.rays == 0 and args.interp == "cic") else None
    missing = ("stale: the trace kernel changed since the last ncu capture" if (args.rays == 0 and args.interp == "cic")
               else "the ncu record covers the full CIC benchmark launch only")
    roof = roofline(total_steps, ms, ck.get("sm_mhz"), fp64_rate, hbm_peak, FIELD_BYTES_BY_SCHEME[args.interp],
                    record, "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s", missing)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, ns, threads, dt = oracle_sample(w, budget_s=args.ref_budget, interp=args.interp)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{ns} seeded rays of the 786,432 ({dt:.1f} s of FP64 oracle work on {threads} threads)"}
    extras = None
    if rank == 0 and ws == 1 and not args.no_extras and args.rays == 0 and args.interp == "cic":
        try:
            extras = run_extras(w, tree, dev)
        except Exception as e:  # the headline line is printed even if a reduced pass fails
            extras = {"error": f"{type(e).__name__}: {e}"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 state / f32 field", "data": "synthetic", "config": dict(workload_config(w), interp=args.interp),
            "steps_per_s": steps_per_s, "rk4_steps_per_step": total_steps,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": args.steps, "clocks": ck, "step_ms_all": times, "wall_s_timed": wall}
    if extras is not None:
        line["extras"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    tree.free()


def run_extras(w, tree, dev):
    """Short, reduced-size passes of the other configurations, reported beside the headline so that
    they are measured in the same run (each with its own clock record):
      * batched: the 64 light cones of the batched configuration at 1/16 of their ray counts in one
        persistent launch (graph replay) against one launch per cone;
      * fp64_field: the FP64-field form on a seeded 1/16 of the benchmark rays, and the largest
        relative difference of the mixed form's outputs from it;
      * tsc: TSC and CIC traces of a seeded quarter of the benchmark rays (time ratio of the schemes);
      * differentiation: 256 x 256 rays of the differentiation workload (128^3 + 3 levels, 10 x 10
        deg to z = 1) on FP32 records: forward, distortion matrix (mixed tangent step) and the mixed
        reverse sweep of the end-point loss (checkpoints every 64 steps)."""
    import torch

    from paper_2111_08744_gb300 import autotune as AT
    from paper_2111_08744_gb300 import binding as B
    from paper_2111_08744_gb300 import inputs as I

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    out = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    # batched light cones (1/16 of the ray counts)
    wb = I.batched_cones(w, n_cones=64, seed=4113, scale=1.0 / 16)
    pb = B.TraceParams.from_workload(wb)
    db = torch.from_numpy(wb.dirs).to(dev)
    g = AT.TraceGraph(tree, pb, db)
    g.replay()
    _, ms_b = timed(g.replay)
    steps_b = int(g.out["n_steps"].sum().item())
    ob = B.alloc_outputs(wb.n_rays, dev)

    def per_cone():
        for c in range(wb.observer.shape[0]):
            lo, hi = int(wb.ray_begin[c]), int(wb.ray_begin[c + 1])
            if hi > lo:
                p1 = B.TraceParams(wb.observer[c:c + 1], wb.z_max[c:c + 1], [0, hi - lo], wb.steps_per_cell,
                                   max_steps=pb.c.max_steps)
                B.trace_rays(tree, p1, db[:, lo:hi].contiguous(), {k: v[..., lo:hi] for k, v in ob.items()})

    _, ms_u = timed(per_cone)
    out["batched"] = {"workload": "64 light cones in the benchmark field, z_max 0.3-2, 1/16 of the ray counts",
                      "n_rays": wb.n_rays, "n_cones": 64, "one_launch_ms": ms_b, "rays_per_s": wb.n_rays / (ms_b * 1e-3),
                      "rk4_steps_per_s": steps_b / (ms_b * 1e-3), "one_launch_per_cone_ms": ms_u}
    del g, ob
    # FP64-field form on a seeded 1/16 of the benchmark rays
    rng = np.random.Generator(np.random.PCG64(5))
    idx = np.sort(rng.choice(w.n_rays, size=w.n_rays // 16, replace=False))
    ws = I.with_rays(w, w.dirs[:, idx])
    t64 = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    ps = B.TraceParams.from_workload(ws)
    ds = torch.from_numpy(ws.dirs).to(dev)
    o64, ms64 = timed(lambda: B.trace_rays(t64, ps, ds))
    o32 = B.trace_rays(tree, ps, ds)
    torch.cuda.synchronize()
    err = {}
    for k, fl in (("x", 1.0), ("chi", 1.0), ("z5", 1e-6), ("d_l", 1.0)):
        r = o64[k].double()
        err[k] = float(((o32[k].double() - r).abs() / r.abs().clamp_min(fl)).max().item())
    steps64 = int(o64["n_steps"].sum().item())
    out["fp64_field"] = {"workload": "the benchmark field with FP64 records, a seeded 1/16 of its rays",
                         "n_rays": int(idx.size), "ms": ms64, "rays_per_s": idx.size / (ms64 * 1e-3),
                         "rk4_steps_per_s": steps64 / (ms64 * 1e-3), "max_rel_diff_mixed_vs_fp64": err}
    t64.free()
    del o64, o32
    # TSC against CIC on the same seeded quarter of the benchmark rays (Table 1 compares the schemes)
    idx4 = np.sort(rng.choice(w.n_rays, size=w.n_rays // 4, replace=False))
    w4 = I.with_rays(w, w.dirs[:, idx4])
    d4 = torch.from_numpy(w4.dirs).to(dev)
    ms_s = {}
    for ip in ("cic", "tsc"):
        p4 = B.TraceParams.from_workload(w4, interp=ip)
        B.trace_rays(tree, p4, d4)
        o4, ms_s[ip] = timed(lambda: B.trace_rays(tree, p4, d4))
        ms_s[ip + "_steps"] = int(o4["n_steps"].sum().item())
        del o4
    out["tsc"] = {"workload": "the benchmark field and a seeded quarter of its rays, TSC (27 cells, neighbour rows "
                              "cached per lane) and CIC", "n_rays": int(idx4.size), "tsc_ms": ms_s["tsc"],
                  "cic_ms": ms_s["cic"], "tsc_over_cic": ms_s["tsc"] / ms_s["cic"],
                  "tsc_rk4_steps_per_s": ms_s["tsc_steps"] / (ms_s["tsc"] * 1e-3),
                  "tsc_effective_GBs": ms_s["tsc_steps"] * FIELD_BYTES_BY_SCHEME["tsc"] / (ms_s["tsc"] * 1e-3) / 1e9}
    # differentiation workload, 256 x 256 rays
    wd = I.cached(I.config_diff, n_pix=256)
    td = B.Octree(wd.box, wd.n_coarse, wd.periodic, wd.slice_eta, I.fp32_levels(wd), wd.bg, "fp32")
    pd = B.TraceParams.from_workload(wd)
    dd = torch.from_numpy(wd.dirs).to(dev)
    ref = B.trace_rays(td, B.TraceParams.from_workload(wd, gravity_on=False), dd)["xi"]
    B.trace_rays(td, pd, dd)
    fwd, ms_f = timed(lambda: B.trace_rays(td, pd, dd))
    _, ms_t = timed(lambda: B.trace_rays_adjoint(td, pd, dd, jacobian=True, lensing=True))
    dxi = 2.0 * (fwd["xi"] - ref)
    _, ms_r = timed(lambda: B.trace_rays_adjoint(td, pd, dd, jacobian=False, lensing=False, dL_dxi=dxi,
                                                 checkpoint_every=64))
    steps_d = int(fwd["n_steps"].sum().item())
    td.free()
    out["differentiation"] = {"workload": "differentiation field (128^3 + 3 levels), 256 x 256 rays over 10 x 10 deg "
                                          "to z = 1, FP32 records", "n_rays": wd.n_rays, "forward_ms": ms_f,
                              "distortion_matrix_ms": ms_t, "reverse_sweep_ms": ms_r,
                              "reverse_over_forward": ms_r / ms_f, "forward_rk4_steps_per_s": steps_d / (ms_f * 1e-3),
                              "reverse_rk4_steps_per_s": steps_d / (ms_r * 1e-3)}
    out["clocks"] = clocks.stop()
    return out


def run_batched(args, ws, rank):
    """Batched light cones: 64 observers in the benchmark field, z_max ~ U[0.3, 2], ray counts
    log-uniform in [1e4, 1e6] (NESTED HEALPix sub-patches); one persistent launch replayed from
    a CUDA graph after the launch-shape autotuner; compared with one launch per cone and with
    the FP64-field form on a ray sample."""
    import torch

    from paper_2111_08744_gb300 import autotune as AT
    from paper_2111_08744_gb300 import binding as B
    from paper_2111_08744_gb300 import build as Bd
    from paper_2111_08744_gb300 import inputs as I

    Bd.build()
    base = I.cached(I.config_amr)
    w = I.batched_cones(base, n_cones=64, seed=4113, scale=args.batched_scale)
    dev = torch.device("cuda", torch.cuda.current_device())
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, I.fp32_levels(w), w.bg, "fp32")
    params = B.TraceParams.from_workload(w)
    dirs = torch.from_numpy(w.dirs).to(dev)
    tune = AT.autotune(tree, params, dirs, sample=262144, repeats=1)
    g = AT.TraceGraph(tree, params, dirs)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(max(0, args.warmup - 1)):
        g.replay()
    torch.cuda.synchronize()
    steps = int(g.out["n_steps"].sum().item())
    ts = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ck = clocks.stop()
    ms = float(np.mean(ts))
    # one launch per cone (same kernel, same launch shape)
    outs = B.alloc_outputs(w.n_rays, dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for c in range(w.observer.shape[0]):
        lo, hi = int(w.ray_begin[c]), int(w.ray_begin[c + 1])
        if hi == lo:
            continue
        p1 = B.TraceParams(w.observer[c:c + 1], w.z_max[c:c + 1], [0, hi - lo], w.steps_per_cell,
                           max_steps=params.c.max_steps)
        B.trace_rays(tree, p1, dirs[:, lo:hi].contiguous(), {k: v[..., lo:hi] for k, v in outs.items()})
    b.record()
    torch.cuda.synchronize()
    ms_unbatched = a.elapsed_time(b)
    # FP64-field form on a seeded 1/16 sample of the rays (accuracy reference and speed)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = np.sort(rng.choice(w.n_rays, size=w.n_rays // 16, replace=False))
    cone = np.searchsorted(w.ray_begin, idx, side="right") - 1
    counts = np.bincount(cone, minlength=w.observer.shape[0])
    ps = B.TraceParams(w.observer, w.z_max, np.concatenate([[0], np.cumsum(counts)]), w.steps_per_cell,
                       max_steps=params.c.max_steps)
    t64 = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    d_s = dirs[:, torch.from_numpy(idx).to(dev)].contiguous()
    a.record()
    o64 = B.trace_rays(t64, ps, d_s)
    b.record()
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b)
    o32 = {k: v[..., torch.from_numpy(idx).to(dev)] for k, v in g.out.items()}
    err = {}
    for k, fl in (("x", 1.0), ("z5", 1e-6), ("chi", 1.0), ("d_l", 1.0)):
        r = o64[k].double()
        err[k] = float(((o32[k].double() - r).abs() / r.abs().clamp_min(fl)).max().item())
    steps64 = int(o64["n_steps"].sum().item())
    line = {"metric": "rays/s, batched light cones (64 observers, z_max 0.3-2) in one persistent launch",
            "value": w.n_rays / (ms * 1e-3), "unit": "rays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 state / f32 field", "data": "synthetic",
            "config": {"workload": "64 light cones in the AMR 256^3 + 3 levels field", "n_rays": w.n_rays,
                       "n_cones": int(w.observer.shape[0]), "rk4_steps": steps, "launch": tune["best"],
                       "graph": True},
            "steps_per_s": steps / (ms * 1e-3), "autotune_ms": tune["ms"],
            "unbatched_ms": ms_unbatched, "unbatched_rays_per_s": w.n_rays / (ms_unbatched * 1e-3),
            "fp64_field_sample": {"rays": int(idx.size), "ms": ms64, "steps_per_s": steps64 / (ms64 * 1e-3),
                                  "max_rel_err_fp32_vs_fp64": err},
            "clocks": ck, "gpu_launches": args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    t64.free()
    tree.free()


def run_large(args, ws, rank):
    """The largest configuration: 1024^3 coarse grid in 2.6 h^-1 Gpc + 4 levels (3 % of the
    volume, 1/8 per level), four time slices (z = 2, 1, 0.5, 0), FP32 records (~135 GB, built on
    the GPU and borrowed by the octree), 50,331,648 HEALPix rays (nside 2048) to z = 2."""
    import torch

    from paper_2111_08744_gb300 import binding as B
    from paper_2111_08744_gb300 import build as Bd
    from paper_2111_08744_gb300 import inputs as I

    Bd.build()
    t0 = time.perf_counter()
    kw = {}
    if args.large_n:
        kw = {"n": args.large_n, "box": 2600.0 * args.large_n / 1024, "nside": args.large_nside}
    w = I.config_large_gpu(**kw)
    t_gen = time.perf_counter() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp32", residency=B.MT_DEVICE_BORROW)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    cells, nbytes = tree.info()
    params = B.TraceParams.from_workload(w)
    dirs = torch.from_numpy(w.dirs).to(dev)
    n = w.n_rays
    out = B.alloc_outputs(n, dev)
    for _ in range(args.warmup):
        B.trace_rays(tree, params, dirs, out)
    torch.cuda.synchronize()
    ts = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for i in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        B.trace_rays(tree, params, dirs, out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ck = clocks.stop()
    st = tree.device_status()
    steps = int(out["n_steps"].sum().item())
    status = torch.bincount(out["status"].long(), minlength=4).tolist()
    levels = torch.bincount(out["level"].long() + 1, minlength=6).tolist()
    ms = float(np.mean(ts))
    tangent = None
    if args.large_tangent:
        # the distortion matrix on every ray: one forward-mode pass (mixed tangent step)
        del out
        torch.cuda.empty_cache()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = B.trace_rays_adjoint(tree, params, dirs, jacobian=True, lensing=True)
        b.record()
        torch.cuda.synchronize()
        tms = a.elapsed_time(b)
        tsteps = int(res["n_steps"].sum().item())
        lens = res["lens"]
        ok = res["status"] == 0
        tangent = {"ms": tms, "rays_per_s": n / (tms * 1e-3), "rk4_steps_per_s": tsteps / (tms * 1e-3),
                   "same_steps_as_trace": tsteps == steps, "device_status": tree.device_status(),
                   "rms_kappa": float(lens[0][ok].pow(2).mean().sqrt()),
                   "rms_gamma": float((lens[1][ok].pow(2) + lens[2][ok].pow(2)).mean().sqrt()),
                   "rms_omega": float(lens[3][ok].pow(2).mean().sqrt())}
        del res
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the ncu record's per-step counts belong to the benchmark workload, not to this one
    roof = roofline(steps, ms, ck.get("sm_mhz"), B.probe_fp64_fma_rate(), hbm, FIELD_BYTES_PER_STEP, None,
                    "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                    "the ncu record covers the benchmark workload only")
    line = {"metric": "rays/s to z=2, largest AMR configuration", "value": n / (ms * 1e-3), "unit": "rays/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 state / f32 field", "data": "synthetic",
            "config": {"workload": w.name, "n_rays": n, "cells_per_level": cells, "device_bytes_octree": nbytes,
                       "n_slices": w.n_slices, "z_max": float(w.z_max[0])},
            "steps_per_s": steps / (ms * 1e-3), "rk4_steps_per_step": steps,
            "roofline": roof,
            "generation_s": t_gen, "build_s": t_build, "device_status": st, "ray_status_counts": status,
            "end_level_counts": levels[1:], "clocks": ck, "step_ms_all": ts, "gpu_launches": args.steps}
    if tangent is not None:
        line["distortion_matrix"] = tangent
    if rank == 0:
        print(json.dumps(line), flush=True)
    tree.free()


def run_diff(args, ws, rank):
    """Differentiation: 1024 x 1024 rays over 10 x 10 deg to z = 1 through the 128^3 + 3 levels
    field; timings of the forward trace, the forward-mode distortion matrix and the reverse-mode
    gradient of L = sum |xi - xi_FLRW|^2 with respect to the records and to phi_0, on the FP32 copy of
    the records (mixed step: FP32 stages, FP64 state) and on the FP64 records (the FP64 reverse sweep
    on a seeded 1/16 of the rays unless --diff-fp64-reverse)."""
    import torch

    from paper_2111_08744_gb300 import binding as B
    from paper_2111_08744_gb300 import build as Bd
    from paper_2111_08744_gb300 import inputs as I

    Bd.build()
    w = I.cached(I.config_diff, n_pix=args.diff_pix)
    dev = torch.device("cuda", torch.cuda.current_device())
    params = B.TraceParams.from_workload(w)
    dirs = torch.from_numpy(w.dirs).to(dev)
    n = w.n_rays

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    # reference end points: the same rays traced without gravity (FLRW)
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    ref = B.trace_rays(tree, B.TraceParams.from_workload(w, gravity_on=False), dirs)["xi"]
    # FP64 records: forward, distortion matrix, reverse sweep (on a sample of the rays by default)
    out, _ = timed(lambda: B.trace_rays(tree, params, dirs))
    out, ms_fwd = timed(lambda: B.trace_rays(tree, params, dirs))
    steps = int(out["n_steps"].sum().item())
    tan, ms_tan = timed(lambda: B.trace_rays_adjoint(tree, params, dirs, jacobian=True, lensing=True))
    dxi = 2.0 * (tan["xi"] - ref)
    lens = tan["lens"]
    if args.diff_fp64_reverse:
        sub = torch.arange(n, device=dev)
    else:
        rng = np.random.Generator(np.random.PCG64(4114))
        sub = torch.from_numpy(np.sort(rng.choice(n, size=n // 16, replace=False))).to(dev)
    p_sub = B.TraceParams(w.observer, w.z_max, [0, int(sub.numel())], w.steps_per_cell,
                          max_steps=params.c.max_steps)
    d_sub = dirs[:, sub].contiguous()
    adj, ms_adj64 = timed(lambda: B.trace_rays_adjoint(tree, p_sub, d_sub, jacobian=False, lensing=False,
                                                       dL_dxi=dxi[:, sub].contiguous(), checkpoint_every=64))
    steps_sub = int(adj["n_steps"].sum().item())
    g0_64, ms_pb = timed(lambda: B.pullback_coarse_phi(tree, adj["dL_drec"], w.slice_weight, w.n_coarse))
    del adj
    tree.free()
    # FP32 copy of the records: mixed trace, mixed tangent, mixed reverse sweep on every ray
    tree32 = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, I.fp32_levels(w), w.bg, "fp32")
    B.trace_rays(tree32, params, dirs)
    out32, ms_fwd32 = timed(lambda: B.trace_rays(tree32, params, dirs))
    steps32 = int(out32["n_steps"].sum().item())
    tan32, ms_tan32 = timed(lambda: B.trace_rays_adjoint(tree32, params, dirs, jacobian=True, lensing=True))
    dA = (tan32["jac"] - tan["jac"]).abs()
    dk = (tan32["lens"][0] - lens[0]).abs()
    dxi32 = 2.0 * (tan32["xi"] - ref)
    rev = {}
    for ce in args.diff_checkpoints:
        adj32, ms = timed(lambda: B.trace_rays_adjoint(tree32, params, dirs, jacobian=False, lensing=False,
                                                       dL_dxi=dxi32, checkpoint_every=ce))
        rev[ce] = ms
    g0_32, _ = timed(lambda: B.pullback_coarse_phi(tree32, adj32["dL_drec"], w.slice_weight, w.n_coarse))
    # the mixed reverse sweep on the sampled rays, against the FP64 one on the same rays
    adj32s = B.trace_rays_adjoint(tree32, p_sub, d_sub, jacobian=False, lensing=False,
                                  dL_dxi=dxi[:, sub].contiguous(), checkpoint_every=64)
    g0_32s = B.pullback_coarse_phi(tree32, adj32s["dL_drec"], w.slice_weight, w.n_coarse)
    torch.cuda.synchronize()
    rel_grad = float((g0_32s - g0_64).norm() / g0_64.norm())
    ck = clocks.stop()
    best_ce = min(rev, key=rev.get)
    mixed = {"forward_ms": ms_fwd32, "tangent_ms": ms_tan32, "reverse_ms_by_checkpoint_interval": rev,
             "forward_steps_per_s": steps32 / (ms_fwd32 * 1e-3),
             "tangent_steps_per_s": steps32 / (ms_tan32 * 1e-3),
             "reverse_steps_per_s": steps32 / (rev[best_ce] * 1e-3),
             "reverse_over_forward": rev[best_ce] / ms_fwd32,
             "jac_abs_diff_vs_fp64_max": float(dA.max()), "jac_abs_diff_vs_fp64_median": float(dA.median()),
             "kappa_abs_diff_median": float(dk.median()),
             "kappa_abs_diff_p99": float(torch.quantile(dk[:1 << 20], 0.99)),
             "grad_phi0_rel_l2_diff_vs_fp64_sample": rel_grad,
             "grad_phi0_rms": float(g0_32.std().item())}
    tree32.free()
    line = {"metric": "differentiable ray tracing: forward, distortion matrix and gradient time",
            "value": n / (rev[best_ce] * 1e-3), "unit": "rays/s (reverse sweep, mixed)", "n_gpus": ws,
            "steps": 1, "warmup": 1, "ms_per_step": rev[best_ce], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 state / f32 field", "data": "synthetic",
            "config": {"workload": w.name, "n_rays": n, "rk4_steps": steps, "checkpoint_every": best_ce},
            "mixed_fp32_field": mixed,
            "fp64_field": {"forward_ms": ms_fwd, "tangent_ms": ms_tan, "forward_steps_per_s": steps / (ms_fwd * 1e-3),
                           "tangent_steps_per_s": steps / (ms_tan * 1e-3), "reverse_rays": int(sub.numel()),
                           "reverse_ms": ms_adj64, "reverse_steps_per_s": steps_sub / (ms_adj64 * 1e-3),
                           "pullback_ms": ms_pb},
            "kappa_rms": float(lens[0].std().item()), "gamma_rms": float(lens[1:3].std().item()),
            "omega_rms": float(lens[3].std().item()), "loss": float(((tan["xi"] - ref) ** 2).sum().item()),
            "clocks": ck, "gpu_launches": 8 + 2 * len(rev)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reduced passes of the batched, FP64-field and differentiation configurations")
    ap.add_argument("--rays", type=int, default=0, help="trace a seeded subset of N rays (profiling only)")
    ap.add_argument("--workload", default="amr", choices=["amr", "batched", "large", "diff"],
                    help="amr: the headline benchmark; batched: 64 light cones (separate report)")
    ap.add_argument("--batched-scale", type=float, default=1.0)
    ap.add_argument("--large-n", type=int, default=0, help="coarse size of a reduced large run (0: 1024)")
    ap.add_argument("--large-nside", type=int, default=2048)
    ap.add_argument("--large-tangent", action="store_true",
                    help="large workload: also time the distortion-matrix pass on every ray")
    ap.add_argument("--diff-pix", type=int, default=1024)
    ap.add_argument("--diff-fp64-reverse", action="store_true",
                    help="diff workload: FP64 reverse sweep on every ray (default: a seeded 1/16)")
    ap.add_argument("--diff-checkpoints", type=int, nargs="+", default=[64, 16],
                    help="diff workload: checkpoint intervals of the mixed reverse sweep to time")
    ap.add_argument("--interp", default="cic", choices=["cic", "ngp", "tsc"],
                    help="amr workload: interpolation scheme (Sect. 2.2; the benchmark line is CIC)")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batched":
        run_batched(args, ws, rank)
    elif args.workload == "large":
        run_large(args, ws, rank)
    elif args.workload == "diff":
        run_diff(args, ws, rank)
    else:
        run_ours(args, ws, rank)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
