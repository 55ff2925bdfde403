"""Launch-shape autotuner and CUDA-graph replay for the trace kernel.

`autotune(tree, params, dirs)` times mt_trace_rays on a seeded sample of the rays for each
candidate (threads per block, blocks per SM, ray ids a warp claims per refill, staging of the CIC
neighbourhood in shared memory or direct loads), keeps the fastest on the octree
(mt_set_launch_config, mt_set_trace_options) and caches the choice in a JSON file keyed by the
device name and a workload signature.  Results do not depend on these choices, only the time does.

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

# (threads per block, blocks per SM, ray chunk, staging: 1 shared-memory neighbourhood, 2 direct loads)
CANDIDATES = [(128, 4, 32, 1), (128, 3, 32, 1), (64, 8, 32, 1), (256, 2, 32, 1), (256, 1, 32, 1),
              (128, 4, 64, 1), (128, 4, 128, 1), (128, 4, 32, 2), (64, 8, 32, 2), (256, 2, 32, 2)]


def _apply(tree, cand):
    bs, bps = cand[0], cand[1]
    chunk, staging = (cand[2], cand[3]) if len(cand) > 2 else (0, 0)
    tree.set_launch_config(bs, bps)
    tree.set_trace_options(chunk, staging)


def _signature(tree: B.Octree, params: B.TraceParams, n_rays: int) -> str:
    cells, nbytes = tree.info()
    return f"{torch.cuda.get_device_name()}|{tree.precision}|{cells}|{n_rays}|{params.c.n_cones}"


def autotune(tree: B.Octree, params: B.TraceParams, dirs: torch.Tensor, sample: int = 131072, repeats: int = 2,
             cache_path: str | None = None, candidates=CANDIDATES, seed: int = 0):
    """Pick the fastest configuration on a sample of the rays; returns {"best": (block, bps, chunk, staging),
    "ms": {...}}."""
    n = int(dirs.shape[1])
    key = _signature(tree, params, n)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            _apply(tree, tuple(cache[key]["best"]))
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
    for cand in candidates:
        _apply(tree, cand)
        B.trace_rays(tree, sp, sd, out)
        ts = []
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            B.trace_rays(tree, sp, sd, out)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        times["x".join(str(v) for v in cand)] = float(np.median(ts))
    best_key = min(times, key=times.get)
    best = tuple(int(v) for v in best_key.split("x"))
    _apply(tree, best)
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
