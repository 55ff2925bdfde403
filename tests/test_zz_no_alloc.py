"""mt_trace_rays_noalloc (a library interface with no counterpart in the paper) against
mt_trace_rays, through the C ABI.

The entry point is for callers that must not allocate GPU memory, e.g. code running
inside an application whose device memory belongs to another allocator, or loops that
cannot afford cudaMalloc's device-wide synchronisation.  Its scratch is a static device
array shared by all calls, so two calls in a row check that the state one call leaves
behind (queue counter, cone table) does not leak into the next.  This file is collected
last so a failure here does not stop the rest of the GPU suite from running first.
"""
import ctypes

import numpy as np
import pytest

from paper_2111_08744_gb300 import binding as B
from paper_2111_08744_gb300 import inputs as I
from tests.gpu_common import compare

pytestmark = pytest.mark.gpu


def _workload():
    w = I.config_amr(n=32, box=250.0, n_levels=2, f1=0.05, ratio=0.3, nside=8, z_max=0.4, seed=17,
                     name="noalloc_amr32")
    return w


def _cones(w, counts, seed=3):
    import dataclasses
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = np.asarray(counts, dtype=np.int64)
    obs = rng.uniform(0.0, w.box, size=(counts.size, 3))
    zm = rng.uniform(0.05, 0.4, size=counts.size)
    dirs = I.healpix_directions(8, nest=True)
    dirs = np.ascontiguousarray(np.tile(dirs, (1, int(np.ceil(counts.sum() / dirs.shape[1]))))[:, :counts.sum()])
    begin = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return dataclasses.replace(w, observer=obs, z_max=zm, ray_begin=begin, dirs=dirs)


def _call_noalloc(tree, params, dirs_t, n):
    import torch
    out = B.alloc_outputs(n)
    o = B.ray_out_struct(out)
    code = B.mt_trace_rays_noalloc(tree.handle, ctypes.byref(params.c), dirs_t.data_ptr(), n, ctypes.byref(o),
                                   torch.cuda.current_stream().cuda_stream)
    return code, out


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_trace_rays_on_two_calls_in_a_row(precision):
    import torch
    w = _cones(_workload(), [200, 0, 57, 300])
    tree = B.Octree.from_workload(w, precision)
    params = B.TraceParams.from_workload(w)
    dirs = torch.from_numpy(w.dirs).cuda()
    n = w.n_rays
    ref = _host(B.trace_rays(tree, params, dirs))
    for _ in range(2):
        code, out = _call_noalloc(tree, params, dirs, n)
        assert code == B.MT_OK, B.status_str(code)
        torch.cuda.synchronize()
        got = _host(out)
        compare(got, ref, 1e-6)
    assert tree.device_status() == B.MT_OK
    tree.free()


def test_noalloc_takes_more_cones_than_kernel_parameters_and_rejects_too_many():
    import torch
    w = _cones(_workload(), np.full(300, 3), seed=5)
    tree = B.Octree.from_workload(w, "fp64")
    dirs = torch.from_numpy(w.dirs).cuda()
    code, out = _call_noalloc(tree, B.TraceParams.from_workload(w), dirs, w.n_rays)
    assert code == B.MT_OK, B.status_str(code)
    torch.cuda.synchronize()
    got = _host(out)
    # reference: mt_trace_rays on cones [0, 256) and [256, 300) separately
    parts = []
    for lo, hi in ((0, 256), (256, 300)):
        b0, b1 = w.ray_begin[lo], w.ray_begin[hi]
        p = B.TraceParams(w.observer[lo:hi], w.z_max[lo:hi], w.ray_begin[lo:hi + 1] - b0, w.steps_per_cell,
                          max_steps=B.TraceParams.from_workload(w).c.max_steps)
        parts.append(_host(B.trace_rays(tree, p, torch.from_numpy(w.dirs[:, b0:b1].copy()).cuda())))
    ref = {k: np.concatenate([parts[0][k], parts[1][k]], axis=-1) for k in parts[0]}
    compare(got, ref, 1e-6)
    # beyond the static table: rejected before any GPU work
    too_many = B.MT_NOALLOC_MAX_CONES + 1
    p = B.TraceParams(np.zeros((too_many, 3)), np.zeros(too_many), np.zeros(too_many + 1, dtype=np.int64))
    code, _ = _call_noalloc(tree, p, dirs[:, :0], 0)
    assert code == B.MT_ERR_UNSUPPORTED
    assert tree.device_status() == B.MT_OK
    tree.free()
