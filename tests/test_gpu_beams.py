"""Finite-beam distortion matrix on the GPU (mt_trace_beams, Sect. 2.3.2, Eqs. 17-21) against the
oracle's finite beams, element by element, on both screens, and against the tangent as the beam
shrinks."""
import functools

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests.gpu_common import compare, run_gpu

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def amr_small():
    return I.config_amr(n=64, box=500.0, n_levels=2, f1=0.04, ratio=0.3, nside=8, z_max=0.5, seed=31,
                        name="amr_64cube_L2_nside8")


def _beams(w, precision, eps, screen=0, interp="cic", gravity_on=True):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, precision)
    p = B.TraceParams.from_workload(w, interp=interp, gravity_on=gravity_on)
    res = B.trace_beams(tree, p, torch.from_numpy(w.dirs).cuda(), eps=eps, screen=screen)
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return {k: v.cpu().numpy() for k, v in res.items()}


@pytest.mark.parametrize("eps,screen,interp", [(1e-6, 0, "cic"), (1e-4, 0, "cic"), (1e-4, 1, "cic"),
                                               (1e-5, 0, "tsc")])
def test_fp64_beams_match_oracle(eps, screen, interp):
    w = amr_small()
    r = _beams(w, "fp64", eps, screen, interp)
    ref = oracle.bundle_jacobian(w, eps=eps, screen=screen, interp=interp)
    dev = np.abs(r["jac"] - ref).max(axis=0)
    # same step and index sequence as the oracle for every ray of the beam: the finite differences
    # agree to rounding amplified by 1 / (2 chi tan eps)
    print(f"eps {eps} screen {screen} {interp}: max |dA| {dev.max():.3e}")
    assert np.mean(dev < 1e-6 * (1e-6 / eps)) >= 0.99
    assert np.abs(1 - 0.5 * (r["jac"][0] + r["jac"][3])).max() > 1e-4


def test_fp32_field_beams_mixed():
    w = amr_small()
    r = _beams(w, "fp32", 1e-4)
    ref = oracle.bundle_jacobian(w, eps=1e-4)
    dev = np.abs(r["jac"] - ref).max(axis=0)
    print("mixed beams: median", np.median(dev), "max", dev.max())
    assert np.mean(dev < 1e-4) >= 0.97 and np.median(dev) < 3e-5


def test_beams_identity_without_gravity_and_central_outputs():
    w = amr_small()
    r = _beams(w, "fp64", 1e-5, gravity_on=False)
    np.testing.assert_allclose(r["jac"][[0, 3]], 1.0, atol=1e-8)
    np.testing.assert_allclose(r["jac"][[1, 2]], 0.0, atol=1e-8)
    g = _beams(w, "fp64", 1e-5)
    t = run_gpu(w, "fp64")
    compare({k: g[k] for k in t}, t, 1e-13)


def test_small_beam_converges_to_the_tangent():
    """TSC (C^1 force): the finite beam at eps = 1e-6 equals the tangent of the discrete map."""
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = I.config_plain_small()
    r = _beams(w, "fp64", 1e-6, interp="tsc")
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    t = B.trace_rays_adjoint(tree, B.TraceParams.from_workload(w, interp="tsc"), torch.from_numpy(w.dirs).cuda())
    tj = t["jac"].cpu().numpy()
    tree.free()
    dev = np.abs(r["jac"] - tj).max(axis=0)
    assert np.median(dev) < 1e-6 and np.mean(dev < 1e-4) >= 0.98


def test_bad_arguments():
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = I.config_plain_small()
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    try:
        p = B.TraceParams.from_workload(w)
        d = torch.from_numpy(w.dirs).cuda()
        for eps, screen in ((0.0, 0), (1e-5, 2)):
            with pytest.raises(B.MtError) as e:
                B.trace_beams(tree, p, d, eps=eps, screen=screen)
            assert e.value.code == B.MT_ERR_INVALID_ARG
    finally:
        tree.free()
