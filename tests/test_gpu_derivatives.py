"""GPU tangent (distortion matrix) and adjoint (gradient with respect to the gridded potential)
against the FP64 oracle: finite beams of Eqs. (17)-(21), closed forms, and central finite
differences of the oracle's end points."""
import functools

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _gpu(w, precision="fp64", dirs=None, **kw):
    import torch
    from paper_2111_08744_gb300 import binding as B
    d = w.dirs if dirs is None else dirs
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, precision)
    p = B.TraceParams.from_workload(w, ray_begin=np.array([0, d.shape[1]]) if dirs is not None else None,
                                    gravity_on=kw.pop("gravity_on", True))
    res = B.trace_rays_adjoint(tree, p, torch.from_numpy(np.ascontiguousarray(d)).cuda(), **kw)
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    out = {}
    for k, v in res.items():
        out[k] = [t.cpu().numpy() for t in v] if isinstance(v, list) else v.cpu().numpy()
    return out


def quadratic_fn(Q, x0):
    Q = np.asarray(Q, dtype=np.float64)

    def fn(xc):
        d = xc - np.asarray(x0, dtype=np.float64)[:, None]
        rec = np.empty((xc.shape[1], 4))
        rec[:, 0] = 0.5 * np.einsum("in,ij,jn->n", d, Q, d)
        rec[:, 1:] = (Q @ d).T
        return rec

    return fn


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_tangent_is_identity_without_gravity(precision, tol):
    w = I.config_plain_small()
    r = _gpu(w, precision, dirs=np.ascontiguousarray(w.dirs[:, ::17]), gravity_on=False)
    np.testing.assert_allclose(r["jac"][[0, 3]], 1.0, atol=tol)
    np.testing.assert_allclose(r["jac"][[1, 2]], 0.0, atol=tol)
    np.testing.assert_allclose(r["lens"][:4], 0.0, atol=tol)
    np.testing.assert_allclose(r["lens"][4], 1.0, atol=2 * tol)


def test_tangent_matches_closed_form_for_quadratic_potential():
    """Same closed form as the oracle pin: A = M - (chi^2/3)(Q_ab - Q_nn delta_ab)."""
    n, box = 16, 4000.0
    xo = np.array([2000.0, 2000.0, 2000.0])
    Q = np.array([[4e-10, 1e-10, 0.0], [1e-10, -2e-10, 0.5e-10], [0.0, 0.5e-10, 1e-10]])
    lv = [H.coarse_level_from_fn(n, box, quadratic_fn(Q, xo))]
    dirs = I.healpix_directions(2)
    w = H.workload(lv, box, n, dirs, z_max=0.45, periodic=0, steps_per_cell=8, observer=xo)
    r = _gpu(w)
    A = r["jac"]
    ref = oracle.bundle_jacobian(w, eps=1e-5)
    scale = r["chi"].max() ** 2 / 3.0 * np.abs(Q).max()
    assert np.abs(A - ref).max() < 0.01 * scale


@functools.lru_cache(maxsize=None)
def _plain_beam():
    w = I.config_plain_small()
    dirs = np.ascontiguousarray(w.dirs[:, 5::48])
    return w, dirs


@pytest.mark.parametrize("precision,tol", [("fp64", 3e-5), ("fp32", 3e-4)])
def test_tangent_matches_oracle_finite_beam(precision, tol):
    """Eq. (21) with a small beam converges to the tangent of the discrete map."""
    w, dirs = _plain_beam()
    r = _gpu(w, precision, dirs=dirs)
    ref = oracle.bundle_jacobian(w, dirs=dirs, eps=1e-6)
    dev = np.abs(r["jac"] - ref)
    # the beam's rays may cross a CIC cell face the central ray does not: allow 2 % outliers
    frac_bad = np.mean(dev.max(axis=0) > tol)
    assert frac_bad <= 0.02, (np.sort(dev.max(axis=0))[-5:], frac_bad)
    assert np.median(dev) < tol / 10
    assert np.abs(1 - 0.5 * (r["jac"][0] + r["jac"][3])).max() > 1e-4    # lensing is present
    # Eq. (11) decomposition round trip
    k, g1, g2, om, det = r["lens"]
    Rm = np.array([[np.cos(om), -np.sin(om)], [np.sin(om), np.cos(om)]])
    S = np.array([[1 - k - g1, -g2], [-g2, 1 - k + g1]])
    A = np.einsum("ijn,jkn->ikn", Rm, S)
    np.testing.assert_allclose(A.reshape(4, -1), r["jac"], atol=1e-12)
    np.testing.assert_allclose(det, r["jac"][0] * r["jac"][3] - r["jac"][1] * r["jac"][2], atol=1e-14)


def test_tangent_pass_outputs_equal_trace():
    from tests.gpu_common import compare, run_gpu
    w, dirs = _plain_beam()
    r = _gpu(w, dirs=dirs)
    t = run_gpu(w, "fp64", dirs=dirs)
    compare({k: r[k] for k in t}, t, 1e-12)


@functools.lru_cache(maxsize=None)
def _amr_beam():
    """Two refinement levels and two time slices: level fallback, phi_eta, the eta slope of
    grad phi and H(eta) all enter the tangent."""
    return I.config_amr(n=32, box=400.0, n_levels=2, f1=0.1, ratio=0.3, nside=4, z_max=0.2, seed=47,
                        name="tan_amr32")


def _beam_directions(dirs, eps):
    """The four beam rays of Eqs. (17)-(20) around each direction (+-tan(eps) along e_1, e_2)."""
    out = np.empty((3, 4 * dirs.shape[1]))
    for i, r in enumerate(dirs.T):
        t1, t2 = np.arctan2(r[1], r[0]), np.arccos(np.clip(r[2], -1.0, 1.0))
        e1 = np.array([-np.sin(t1), np.cos(t1), 0.0])
        e2 = np.array([-np.cos(t1) * np.cos(t2), -np.sin(t1) * np.cos(t2), np.sin(t2)])
        for j, (e, sg) in enumerate(((e1, 1), (e1, -1), (e2, -1), (e2, 1))):
            d = r + sg * np.tan(eps) * e
            out[:, 4 * i + j] = d / np.linalg.norm(d)
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 3e-5), ("fp32", 3e-4)])
def test_tangent_matches_oracle_finite_beam_amr(precision, tol):
    w = _amr_beam()
    eps = 1e-6
    r = _gpu(w, precision)
    ref = oracle.bundle_jacobian(w, eps=eps)
    dev = np.abs(r["jac"] - ref).max(axis=0)
    # a beam ray whose step sequence differs from the central ray's (it changes AMR level at a
    # different step, so its step size jumps) makes the finite difference no derivative: such
    # rays are reported, the others judged
    steps_c = oracle.trace(w)["n_steps"]
    steps_b = oracle.trace(w, dirs=_beam_directions(w.dirs, eps))["n_steps"].reshape(-1, 4)
    smooth = (steps_b == steps_c[:, None]).all(axis=1)
    print("rays with a step-count change inside the beam:", int((~smooth).sum()), "of", smooth.size)
    assert smooth.mean() > 0.8
    frac_bad = np.mean(dev[smooth] > tol)
    assert frac_bad <= 0.03, (np.sort(dev[smooth])[-5:], frac_bad)
    assert np.median(dev) < tol / 10, np.median(dev)
    assert np.abs(1 - 0.5 * (r["jac"][0] + r["jac"][3])).max() > 1e-4


def test_mixed_tangent_matches_fp64_tangent_on_the_same_records():
    """FP32 field with the mixed tangent step against the FP64 tangent of the same (rounded) records."""
    import dataclasses
    w = _amr_beam()
    lv = [I.Level(l.keys, l.records.astype(np.float32).astype(np.float64)) for l in w.levels]
    w32 = dataclasses.replace(w, levels=lv)
    a = _gpu(w32, "fp64")
    b = _gpu(w32, "fp32")
    dev = np.abs(a["jac"] - b["jac"])
    print("mixed vs fp64 tangent: max", dev.max(), "median", np.median(dev))
    assert np.median(dev) < 1e-6
    assert np.mean(dev.max(axis=0) > 1e-4) <= 0.02
    dl = np.abs(a["lens"][:3] - b["lens"][:3])
    assert np.median(dl) < 1e-6


def test_mixed_tangent_pass_outputs_equal_mixed_trace():
    """The mixed tangent pass advances each ray as the mixed trace does (same step and level
    sequence; the two kernels round their FP32 stage arithmetic independently)."""
    from tests.gpu_common import compare, run_gpu
    w = _amr_beam()
    r = _gpu(w, "fp32")
    t = run_gpu(w, "fp32")
    compare({k: r[k] for k in t}, t, 1e-6)


# ----------------------------------------------------------------------------- adjoint

@functools.lru_cache(maxsize=None)
def _adj_workload():
    w = I.config_amr(n=16, box=200.0, n_levels=1, f1=0.1, ratio=0.3, nside=2, z_max=0.1, seed=41,
                     name="adj_amr16")
    return w


def _loss_and_xi(w, out):
    es = oracle.eta_stop(w.bg, float(w.z_max[0]))
    xi = oracle.xi_on_surface(out, es)
    ref = w.observer[0][:, None] + w.dirs * (w.bg[-1, 0] - es)
    return float(((xi - ref) ** 2).sum()), xi - ref


def _near_path_rows(w, lev, radius_cells, seed, count):
    """Seeded rows of level `lev` whose cells lie within radius_cells (max norm, periodic) of some
    ray's straight path to the stop distance: records a ray can use (chosen from the geometry alone)."""
    es = oracle.eta_stop(w.bg, float(w.z_max[0]))
    chi = (w.bg[-1, 0] - es) * 1.01
    dxl = w.box / (w.n_coarse << lev)
    ci, cj, ck = I._demorton(w.levels[lev].keys)
    xc = (np.stack([ci, cj, ck]).astype(np.float64) + 0.5) * dxl
    s = np.arange(0.0, chi + dxl, 0.5 * dxl)
    pts = (w.observer[0][:, None, None] + w.dirs[:, :, None] * s[None, None, :]).reshape(3, -1) % w.box
    near = np.zeros(xc.shape[1], bool)
    for a in range(0, pts.shape[1], 4096):
        q = (xc[:, :, None] - pts[:, None, a:a + 4096] + 0.5 * w.box) % w.box - 0.5 * w.box
        near |= (np.abs(q).max(axis=0) < radius_cells * dxl).any(axis=1)
    rows = np.nonzero(near)[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(rows, size=min(count, rows.size), replace=False)


def _richardson_fd(loss, d):
    """Central differences at d and d/2 combined to cancel the d^2 term; also whether both pairs
    took the same step counts (no decision crossed) and the two quotients."""
    q = []
    same = True
    for dd in (d, 0.5 * d):
        (lp, sp), (lm, sm) = loss(+dd), loss(-dd)
        q.append((lp - lm) / (2 * dd))
        same = same and np.array_equal(sp, sm)
    return (4.0 * q[1] - q[0]) / 3.0, same, q


def test_adjoint_matches_oracle_finite_differences():
    """dL/d(record) for L = sum |xi - xi_FLRW|^2 against central differences of the oracle, on
    seeded records (each level, component and slice) of cells the rays pass."""
    import dataclasses
    import torch
    w = _adj_workload()
    base = _gpu(w)
    _, dxi = _loss_and_xi(w, base)
    r = _gpu(w, jacobian=False, lensing=False, dL_dxi=torch.from_numpy(2.0 * dxi).cuda())
    grads = r["dL_drec"]
    assert all(np.isfinite(g).all() for g in grads)
    picks = []
    for lev in range(len(w.levels)):
        for i, row in enumerate(_near_path_rows(w, lev, 1.0, 100 + lev, 8)):
            picks.append((lev, int(row), i % w.n_slices, i % 4))
    errs, kinked = [], []
    gscale = max(np.abs(g).max() for g in grads)
    for lev, row, sl, comp in picks:
        val = w.levels[lev].records[row, sl, comp]
        g = grads[lev][row, sl, comp]
        rms = np.sqrt((w.levels[lev].records[:, :, comp] ** 2).mean())

        def loss(t):
            lv = [I.Level(l.keys, l.records.copy()) for l in w.levels]
            lv[lev].records[row, sl, comp] = val + t
            o = oracle.trace(dataclasses.replace(w, levels=lv))
            return _loss_and_xi(w, o)[0], o["n_steps"]

        fd, same, q = _richardson_fd(loss, 0.02 * rms)
        floor = 1e-6 * gscale
        # a perturbation that moves a ray across a decision (a step count, a level, or a CIC cell plane
        # where the interpolant's derivative jumps) between the two step sizes makes the quotients
        # disagree: such picks are reported, not judged, and must be few
        if not same or abs(q[0] - q[1]) > 1e-5 * max(abs(fd), floor):
            kinked.append((lev, row, sl, comp, q, g))
            continue
        errs.append(abs(fd - g) / max(abs(fd), floor))
    errs = np.array(errs)
    print("relative errors", errs, "kinked", kinked)
    assert len(kinked) <= len(picks) // 8, kinked
    assert errs.max() < 1e-5, errs


def test_adjoint_checkpoint_interval_does_not_change_gradients():
    import torch
    w = _adj_workload()
    base = _gpu(w)
    _, dxi = _loss_and_xi(w, base)
    g64 = _gpu(w, jacobian=False, lensing=False, dL_dxi=torch.from_numpy(2 * dxi).cuda(), checkpoint_every=64)
    g7 = _gpu(w, jacobian=False, lensing=False, dL_dxi=torch.from_numpy(2 * dxi).cuda(), checkpoint_every=7)
    for a, b in zip(g64["dL_drec"], g7["dL_drec"]):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9 * np.abs(a).max())


def test_pullback_to_coarse_phi_matches_oracle_finite_differences():
    """dL/dphi_0 through the field model (records rebuilt from phi_0 by the generator) against
    central differences of the oracle's loss in seeded coarse cells the rays pass."""
    import dataclasses
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = _adj_workload()
    base = _gpu(w)
    _, dxi = _loss_and_xi(w, base)
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    p = B.TraceParams.from_workload(w)
    res = B.trace_rays_adjoint(tree, p, torch.from_numpy(w.dirs).cuda(), jacobian=False, lensing=False,
                               dL_dxi=torch.from_numpy(2 * dxi).cuda())
    g = B.pullback_coarse_phi(tree, res["dL_drec"], w.slice_weight, w.n_coarse).cpu().numpy()
    tree.free()
    errs, kinked = [], []
    rows = _near_path_rows(w, 0, 1.0, 7, 16)
    for m in rows:
        ci, cj, ck = I._demorton(np.array([m], dtype=np.uint64))
        i, j, k = int(ci[0]), int(cj[0]), int(ck[0])

        def loss(t):
            phi = w.phi0.copy()
            phi[i, j, k] += t
            o = oracle.trace(dataclasses.replace(w, levels=I.records_from_phi0(w, phi)))
            return _loss_and_xi(w, o)[0], o["n_steps"]

        fd, same, q = _richardson_fd(loss, 2e-7)
        floor = 1e-6 * np.abs(g).max()
        if not same or abs(q[0] - q[1]) > 1e-5 * max(abs(fd), floor):
            kinked.append((m, q, g[m]))
            continue
        errs.append(abs(fd - g[m]) / max(abs(fd), floor))
    errs = np.array(errs)
    print("pullback relative errors", errs, "kinked", kinked)
    assert len(kinked) <= len(rows) // 8, kinked
    assert errs.max() < 1e-5, errs


def test_autograd_functions_backpropagate_the_adjoint():
    import torch
    from paper_2111_08744_gb300 import autograd as AG
    from paper_2111_08744_gb300 import binding as B
    w = _adj_workload()
    tc = AG.TraceContext(w, checkpoint_every=16)
    recs = [torch.from_numpy(l.records).cuda().requires_grad_(True) for l in w.levels]
    xi = AG.RayEndpoints.apply(tc, *recs)
    es = oracle.eta_stop(w.bg, float(w.z_max[0]))
    ref = torch.from_numpy(w.observer[0][:, None] + w.dirs * (w.bg[-1, 0] - es)).cuda()
    loss = ((xi - ref) ** 2).sum()
    loss.backward()
    # same as calling the adjoint directly
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")
    res = B.trace_rays_adjoint(tree, B.TraceParams.from_workload(w), torch.from_numpy(w.dirs).cuda(),
                               jacobian=False, lensing=False, dL_dxi=(2 * (xi - ref)).detach(), checkpoint_every=16)
    tree.free()
    for r, g in zip(recs, res["dL_drec"]):
        np.testing.assert_allclose(r.grad.cpu().numpy(), g.cpu().numpy(), rtol=1e-12, atol=1e-30)
    # coarse-phi form: its gradient is the pull-back of the record gradients
    phi0 = torch.from_numpy(w.phi0).cuda().requires_grad_(True)
    xi2 = AG.CoarsePhiEndpoints.apply(tc, phi0)
    np.testing.assert_allclose(xi2.detach().cpu().numpy(), xi.detach().cpu().numpy(), rtol=0, atol=1e-9)
    ((xi2 - ref) ** 2).sum().backward()
    assert torch.isfinite(phi0.grad).all() and phi0.grad.abs().max() > 0
