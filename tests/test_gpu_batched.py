"""Batched light cones in one persistent launch, CUDA-graph replay and the launch-shape
autotuner: results against the oracle, and independence of results from the launch shape."""
import functools

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests.gpu_common import compare

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def batched_small():
    # config-3 shape at reduced size: 64 cones in a 64^3 + 2-level field, z_max ~ U[0.3, 2],
    # ray counts log-uniform in [1e2, 1e4]
    base = I.config_amr(n=64, box=500.0, n_levels=2, f1=0.04, ratio=0.3, nside=1, z_max=1.0, seed=33,
                        name="amr_64cube_L2")
    return I.batched_cones(base, n_cones=64, n_min=1e2, n_max=1e4, seed=4114)


def _run(w, precision, **kw):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = B.Octree.from_workload(w, precision)
    if "launch" in kw:
        launch = kw.pop("launch")
        tree.set_launch_config(*launch[:2])
        if len(launch) > 2:
            tree.set_trace_options(*launch[2:])
    out = B.trace_rays(tree, B.TraceParams.from_workload(w), torch.from_numpy(w.dirs).cuda())
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_batched_cones_match_oracle_on_a_sample():
    w = batched_small()
    assert w.observer.shape[0] == 64 and w.z_max.max() > 1.5
    rng = np.random.Generator(np.random.PCG64(1))
    idx = np.sort(rng.choice(w.n_rays, size=400, replace=False))
    cone = np.searchsorted(w.ray_begin, idx, side="right") - 1
    # oracle on the sample: one cone table per sampled ray
    import dataclasses
    ws = dataclasses.replace(w, observer=w.observer[cone], z_max=w.z_max[cone], dirs=w.dirs[:, idx],
                             ray_begin=np.arange(idx.size + 1, dtype=np.int64))
    ref = oracle.trace(ws)
    got64 = _run(w, "fp64")
    compare(got64, ref, 1e-6, idx=idx)
    got32 = _run(w, "fp32")
    keys = ["x", "eta", "chi", "path", "z0", "z1", "z4", "z5", "d_a", "d_l", "phi_o", "phi_s", "isw"]
    compare(got32, ref, 1e-4, exact_ints=False, idx=idx, keys=keys)


@pytest.mark.parametrize("launch", [(64, 8), (256, 1), (128, 2), (128, 4, 64, 1), (128, 4, 32, 2), (256, 2, 128, 2)])
def test_results_do_not_depend_on_launch_shape(launch):
    """Block size, blocks per SM, the ray chunk a warp claims and the staging of the CIC neighbourhood
    in shared memory change the time only: every output is equal bit for bit."""
    w = batched_small()
    a = _run(w, "fp32")
    b = _run(w, "fp32", launch=launch)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_graph_replay_and_autotuner():
    import torch
    from paper_2111_08744_gb300 import autotune as AT
    from paper_2111_08744_gb300 import binding as B
    w = batched_small()
    tree = B.Octree.from_workload(w, "fp32")
    params = B.TraceParams.from_workload(w)
    dirs = torch.from_numpy(w.dirs).cuda()
    res = AT.autotune(tree, params, dirs, sample=20000, repeats=1)
    assert tuple(res["best"]) in AT.CANDIDATES
    direct = {k: v.clone() for k, v in B.trace_rays(tree, params, dirs).items()}
    g = AT.TraceGraph(tree, params, dirs)
    for _ in range(2):
        out = g.replay()
        torch.cuda.synchronize()
        for k in direct:
            assert torch.equal(out[k], direct[k]), k
    assert tree.device_status() == B.MT_OK
    tree.free()
