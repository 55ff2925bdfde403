"""The GPU-side generator of the large AMR workload (same field model, four time slices) at a
size the oracle checks in full, with the records borrowed by the octree (no copy)."""
import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests.gpu_common import compare

pytestmark = pytest.mark.gpu


def _small_large():
    return I.config_large_gpu(n=32, box=250.0, n_levels=3, f1=0.06, ratio=0.25, nside=4, z_max=1.2,
                              slice_z=(2.0, 1.0, 0.5, 0.0), seed=77)


def _to_host(w):
    lv = []
    for l, L in enumerate(w.levels):
        rec = L.records.double().cpu().numpy()
        keys = np.arange(rec.shape[0], dtype=np.uint64) if L.keys is None else \
            L.keys.cpu().numpy().astype(np.uint64)
        lv.append(I.Level(keys=keys, records=rec))
    import dataclasses
    return dataclasses.replace(w, levels=lv)


def test_gpu_generated_field_traces_like_the_oracle():
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = _small_large()
    assert len(w.levels) == 4 and w.levels[0].records.shape[1] == 4
    counts = [int(L.records.shape[0]) for L in w.levels]
    assert all(c > 0 for c in counts[1:]) and all(c % 8 == 0 for c in counts[1:])
    wh = _to_host(w)
    ref = oracle.trace(wh)
    assert (ref["level"] > 0).any() and (ref["status"] == 0).all()
    dirs = torch.from_numpy(w.dirs).cuda()
    p = B.TraceParams.from_workload(w)
    # FP32 records borrowed from the generator's CUDA tensors
    t32 = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp32", residency=B.MT_DEVICE_BORROW)
    g32 = {k: v.cpu().numpy() for k, v in B.trace_rays(t32, p, dirs).items()}
    torch.cuda.synchronize()
    assert t32.device_status() == B.MT_OK
    keys = ["x", "eta", "chi", "path", "z0", "z1", "z4", "z5", "d_a", "d_l", "phi_o", "phi_s", "isw"]
    compare(g32, ref, 1e-4, exact_ints=False, keys=keys)
    t32.free()
    # the FP64 form of the same (FP32-valued) records is index-exact against the oracle
    t64 = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, wh.levels, w.bg, "fp64")
    g64 = {k: v.cpu().numpy() for k, v in B.trace_rays(t64, p, dirs).items()}
    t64.free()
    compare(g64, ref, 1e-6)
