"""Launch-shape autotuner and CUDA-graph replay for the trace kernel.

`autotune(tree, params, dirs)` times mt_trace_rays on a seeded sample of the rays for each
candidate (threads per block, blocks per SM), keeps the fastest on the octree
(mt_set_launch_config) and caches the choice in a JSON file keyed by the device name and a
workload signature.  Results do not depend on the launch shape, only the time does.

`TraceGraph` captures one mt_trace_rays call (the queue reset and the persistent launch) in
a CUDA graph; `replay()` re-runs it on the same buffers (e.g. after the field or the ray
directions were updated in place).
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import binding as B

CANDIDATES = [(128, 4), (128, 3), (64, 8), (64, 6), (256, 2), (256, 1)]


def _signature(tree: B.Octree, params: B.TraceParams, n_rays: int) -> str:
    cells, nbytes = tree.info()
    return f"{torch.cuda.get_device_name()}|{tree.precision}|{cells}|{n_rays}|{params.c.n_cones}"


def autotune(tree: B.Octree, params: B.TraceParams, dirs: torch.Tensor, sample: int = 131072, repeats: int = 2,
             cache_path: str | None = None, candidates=CANDIDATES, seed: int = 0):
    """Pick the fastest launch shape on a sample of the rays; returns {"best": (block, bps), "ms": {...}}."""
    n = int(dirs.shape[1])
    key = _signature(tree, params, n)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            best = tuple(cache[key]["best"])
            tree.set_launch_config(*best)
            return cache[key]
    # sample: a seeded subset of rays, with the cone table cut accordingly
    rng = np.random.Generator(np.random.PCG64(seed))
    m = min(n, sample)
    idx = np.sort(rng.choice(n, size=m, replace=False))
    begin = params.begin
    cone = np.searchsorted(begin, idx, side="right") - 1
    counts = np.bincount(cone, minlength=len(begin) - 1)
    sp = B.TraceParams(params.obs, params.zmax, np.concatenate([[0], np.cumsum(counts)]), params.c.steps_per_cell,
                       bool(params.c.gravity_on), params.c.max_steps, params.interp)
    sd = dirs[:, torch.from_numpy(idx).to(dirs.device)].contiguous()
    out = B.alloc_outputs(m, dirs.device, names=["n_steps"])
    times = {}
    for bs, bps in candidates:
        tree.set_launch_config(bs, bps)
        B.trace_rays(tree, sp, sd, out)
        ts = []
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            B.trace_rays(tree, sp, sd, out)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        times[f"{bs}x{bps}"] = float(np.median(ts))
    best_key = min(times, key=times.get)
    best = tuple(int(v) for v in best_key.split("x"))
    tree.set_launch_config(*best)
    res = {"best": list(best), "ms": times, "sample_rays": m}
    if cache_path:
        cache[key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res


class TraceGraph:
    """One mt_trace_rays call captured in a CUDA graph (fixed buffers and parameters)."""

    def __init__(self, tree: B.Octree, params: B.TraceParams, dirs: torch.Tensor, out=None):
        self.tree, self.params, self.dirs = tree, params, dirs
        self.out = out if out is not None else B.alloc_outputs(int(dirs.shape[1]), dirs.device)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            B.trace_rays(tree, params, dirs, self.out, stream=side)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            B.trace_rays(tree, params, dirs, self.out, stream=side)

    def replay(self):
        self.graph.replay()
        return self.out
