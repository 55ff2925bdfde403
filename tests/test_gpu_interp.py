"""NGP (Eq. 7) and TSC (Eq. 9) interpolation with the level fallback of Sect. 2.2 on the GPU
against the FP64 oracle: the same bar as CIC (bit-exact step counts, levels and status; relative
1e-6 on the FP64 field, 1e-4 on the FP32 field), the distortion matrix with TSC against the
oracle's finite beams, and the error codes of the unsupported combinations."""
import functools

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests.gpu_common import compare, run_gpu

pytestmark = pytest.mark.gpu

SCHEMES = ["ngp", "tsc"]
MIXED_KEYS = ["x", "eta", "chi", "path", "lambda", "z0", "z1", "z4", "z5", "d_a", "d_l", "phi_o", "phi_s", "isw", "k"]


@functools.lru_cache(maxsize=None)
def amr_small():
    # 64^3 coarse grid (500 h^-1 Mpc) + 2 levels, two slices, 3072 NESTED rays to z = 0.5
    return I.config_amr(n=64, box=500.0, n_levels=2, f1=0.04, ratio=0.3, nside=16, z_max=0.5, seed=31,
                        name="amr_64cube_L2_nside16")


@functools.lru_cache(maxsize=None)
def oracle_of(name, interp):
    w = {"plain": I.config_plain_small, "amr_small": amr_small}[name]()
    return oracle.trace(w, interp=interp)


@pytest.mark.parametrize("interp", SCHEMES)
def test_plain_fp64(interp):
    w = I.config_plain_small()
    compare(run_gpu(w, "fp64", interp=interp), oracle_of("plain", interp), 1e-6)


@pytest.mark.parametrize("interp", SCHEMES)
def test_amr_small_fp64_bit_exact_indices(interp):
    w = amr_small()
    ref = oracle_of("amr_small", interp)
    assert (ref["level"] > 0).any()
    compare(run_gpu(w, "fp64", interp=interp), ref, 1e-6)


def test_amr_small_fp32_field_mixed_precision_tsc():
    w = amr_small()
    got = run_gpu(w, "fp32", interp="tsc")
    ref = oracle_of("amr_small", "tsc")
    compare(got, ref, 1e-4, exact_ints=False, keys=MIXED_KEYS)
    assert np.mean(got["n_steps"] == ref["n_steps"]) > 0.95
    assert np.mean(got["level"] == ref["level"]) > 0.99


def test_amr_small_fp32_field_mixed_precision_ngp():
    """NGP's force is discontinuous at every cell face: where the mixed path's FP32 stage position
    and the oracle's FP64 one fall on two sides of a face (rounding, not a different rule), the ray
    takes a different force for that stage.  Judged per ray: nearly all within the mixed
    tolerance, none far off."""
    from tests.gpu_common import rel_err
    w = amr_small()
    got = run_gpu(w, "fp32", interp="ngp")
    ref = oracle_of("amr_small", "ngp")
    worst = np.zeros(w.n_rays)
    for k in MIXED_KEYS:
        e = rel_err(got[k], ref[k], k)
        worst = np.maximum(worst, e.reshape(-1, w.n_rays).max(axis=0))
    print("ngp mixed: fraction within 1e-4", np.mean(worst <= 1e-4), "max", worst.max())
    assert np.mean(worst <= 1e-4) >= 0.97
    # an end point on the other side of a face reads the neighbouring cell's phi (phi_s, z1, z4):
    # at most a cell-to-cell difference of the potential, a few 1e-2 of it
    assert worst.max() < 0.1
    assert np.mean(got["n_steps"] == ref["n_steps"]) > 0.95


def test_schemes_differ():
    """The three schemes give different trajectories on the same field (the selector is honoured)."""
    w = amr_small()
    xs = [run_gpu(w, "fp64", dirs=np.ascontiguousarray(w.dirs[:, :256]), interp=s)["x"] for s in ("cic", "ngp", "tsc")]
    assert np.abs(xs[0] - xs[1]).max() > 1e-6 and np.abs(xs[0] - xs[2]).max() > 1e-6


def _gpu_tangent(w, precision, dirs, interp):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, precision)
    p = B.TraceParams.from_workload(w, ray_begin=np.array([0, dirs.shape[1]]), interp=interp)
    res = B.trace_rays_adjoint(tree, p, torch.from_numpy(np.ascontiguousarray(dirs)).cuda())
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return {k: v.cpu().numpy() for k, v in res.items()}


@pytest.mark.parametrize("precision,tol", [("fp64", 3e-5), ("fp32", 3e-4)])
def test_tsc_tangent_matches_oracle_finite_beam(precision, tol):
    """With TSC the interpolated force is C^1, so the finite beam converges to the tangent of the
    discrete map with fewer cell-face outliers than CIC."""
    w = I.config_plain_small()
    dirs = np.ascontiguousarray(w.dirs[:, 5::48])
    r = _gpu_tangent(w, precision, dirs, "tsc")
    ref = oracle.bundle_jacobian(w, dirs=dirs, eps=1e-6, interp="tsc")
    dev = np.abs(r["jac"] - ref).max(axis=0)
    print("tsc tangent vs beam: median", np.median(dev), "max", dev.max())
    assert np.mean(dev > tol) <= 0.02
    assert np.median(dev) < tol / 10
    assert np.abs(1 - 0.5 * (r["jac"][0] + r["jac"][3])).max() > 1e-4
    # and against the same field's CIC matrix: the schemes agree to the lensing signal's scale only
    cic = _gpu_tangent(w, precision, dirs, "cic")
    assert np.abs(cic["jac"] - r["jac"]).max() > 1e-6


def test_reverse_mode_rejects_ngp_tsc_and_bad_selector():
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = I.config_plain_small()
    dirs = torch.from_numpy(np.ascontiguousarray(w.dirs[:, :64])).cuda()
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    try:
        p = B.TraceParams.from_workload(w, ray_begin=np.array([0, 64]), interp="tsc")
        with pytest.raises(B.MtError) as e:
            B.trace_rays_adjoint(tree, p, dirs, jacobian=False, lensing=False,
                                 dL_dxi=torch.zeros((3, 64), dtype=torch.float64, device="cuda"))
        assert e.value.code == B.MT_ERR_UNSUPPORTED
        bad = B.TraceParams.from_workload(w, ray_begin=np.array([0, 64]), interp=3)
        with pytest.raises(B.MtError) as e:
            B.trace_rays(tree, bad, dirs)
        assert e.value.code == B.MT_ERR_INVALID_ARG
    finally:
        tree.free()
