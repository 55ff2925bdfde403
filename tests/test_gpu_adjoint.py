"""Reverse mode (record gradients, coarse-phi pull-back) and its forward counterpart (J v) against
each other and against the FP64 oracle.

* Dot-product test: the reverse mode of mt_trace_rays_adjoint applies J^T for the same discrete map
  whose forward derivative mt_trace_rays_jvp applies, so <J v, w> = <v, J^T w> for any record
  perturbation v and end-point cotangent w, to rounding (1e-10 relative).
* J v against central differences of the oracle's end points along v, ray by ray.
* dL/dphi_0 against central differences of the oracle's loss on 64 seeded coarse cells of the
  differentiation workload (128^3 + 3 levels, a 64 x 64 patch of the 10 x 10 deg grid, to z = 1).
"""
import dataclasses
import functools

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _small():
    return I.config_amr(n=16, box=200.0, n_levels=1, f1=0.1, ratio=0.3, nside=2, z_max=0.1, seed=41,
                        name="adj_amr16")


@functools.lru_cache(maxsize=None)
def _diff_patch():
    # the differentiation workload's generator (128^3 in 1 h^-1 Gpc + 3 levels, two slices) with
    # a 64 x 64 tangent-plane patch of 10 x 10 deg traced to z = 1
    return I.cached(I.config_diff, n_pix=64)


def _tree(w):
    from paper_2111_08744_gb300 import binding as B
    return B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, "fp64")


def _direction(w, seed):
    """A random record perturbation, each component scaled to that component's rms."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = []
    for l in w.levels:
        scale = np.sqrt((l.records ** 2).mean(axis=(0, 1)))
        v.append(rng.normal(size=l.records.shape) * scale[None, None, :])
    return v


def _jvp(w, v):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = _tree(w)
    r = B.trace_rays_jvp(tree, B.TraceParams.from_workload(w), torch.from_numpy(w.dirs).cuda(),
                         [torch.from_numpy(x).cuda() for x in v])
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return {k: x.cpu().numpy() for k, x in r.items()}


def _vjp(w, wxi):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = _tree(w)
    r = B.trace_rays_adjoint(tree, B.TraceParams.from_workload(w), torch.from_numpy(w.dirs).cuda(), jacobian=False,
                             lensing=False, dL_dxi=torch.from_numpy(np.ascontiguousarray(wxi)).cuda())
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return [g.cpu().numpy() for g in r["dL_drec"]], r["status"].cpu().numpy()


@pytest.mark.parametrize("which", ["small", "diff_patch"])
def test_adjoint_is_the_transpose_of_the_jvp(which):
    w = _small() if which == "small" else _diff_patch()
    v = _direction(w, 17)
    rng = np.random.Generator(np.random.PCG64(18))
    wxi = rng.normal(size=(3, w.n_rays))
    jv = _jvp(w, v)
    jtw, status = _vjp(w, wxi)
    assert (status == 0).all() and (jv["status"] == 0).all()
    lhs = float((jv["dxi"] * wxi).sum())
    rhs = float(sum((a * b).sum() for a, b in zip(v, jtw)))
    rel = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    print(f"<J v, w> = {lhs:.15e}, <v, J^T w> = {rhs:.15e}, relative difference {rel:.2e}")
    assert abs(lhs) > 0
    assert rel < 1e-10


def test_jvp_matches_oracle_central_differences_ray_by_ray():
    """dxi along v against (xi(rec + e v) - xi(rec - e v)) / 2e of the oracle; Richardson
    extrapolation of e and e/2 removes the e^2 term."""
    w = _small()
    v = _direction(w, 23)
    jv = _jvp(w, v)["dxi"]
    es = oracle.eta_stop(w.bg, float(w.z_max[0]))

    def xi_at(t):
        lv = [I.Level(l.keys, l.records + t * d) for l, d in zip(w.levels, v)]
        o = oracle.trace(dataclasses.replace(w, levels=lv))
        return oracle.xi_on_surface(o, es), o["n_steps"], o["level"]

    fd, same = [], np.ones(w.n_rays, bool)
    for e in (4e-3, 2e-3):
        (xp, sp, lp), (xm, sm, lm) = xi_at(e), xi_at(-e)
        fd.append((xp - xm) / (2 * e))
        same &= (sp == sm) & (lp == lm)
    rich = (4.0 * fd[1] - fd[0]) / 3.0
    scale = np.abs(rich).max()
    norm = np.maximum(np.abs(rich).max(axis=0), 1e-3 * scale)
    # a ray whose perturbed traces cross a decision (a step count, a level, or a CIC cell plane where
    # the interpolant's derivative jumps) between the two step sizes: its two quotients disagree.
    # Such rays are reported, not judged, and must be few.
    smooth = same & (np.abs(fd[0] - fd[1]).max(axis=0) / norm < 1e-5)
    err = np.abs(rich - jv).max(axis=0) / norm
    print("J v vs central differences: max", err[smooth].max(), "median", np.median(err[smooth]),
          "rays judged", smooth.sum(), "of", smooth.size)
    assert smooth.mean() >= 0.8
    assert err[smooth].max() < 1e-5


def _affected_rays(w, cell, radius_cells):
    """Rays whose straight path to the stop distance passes within radius_cells coarse cells (max
    norm, periodic) of the centre of coarse cell `cell`: the only rays a change of phi_0 there can
    move (5-point stencil, trilinear prolongation and CIC together reach 4 cells)."""
    dx = w.box / w.n_coarse
    c = (np.asarray(cell, dtype=np.float64) + 0.5) * dx
    es = oracle.eta_stop(w.bg, float(w.z_max[0]))
    chi = (w.bg[-1, 0] - es) * 1.01
    s = np.arange(0.0, chi + dx, 0.5 * dx)
    hit = np.zeros(w.n_rays, bool)
    for a in range(0, w.n_rays, 512):
        d = w.dirs[:, a:a + 512]
        p = w.observer[0][:, None, None] + d[:, :, None] * s[None, None, :]
        q = (p - c[:, None, None] + 0.5 * w.box) % w.box - 0.5 * w.box
        hit[a:a + 512] = (np.abs(q).max(axis=0) < radius_cells * dx).any(axis=1)
    return np.nonzero(hit)[0]


def _impulse_records(w, cell):
    """Records of the field model for phi_0 = the unit impulse at `cell` (no detail terms): the
    linear part of inputs.records_from_phi0, evaluated only where it is non-zero."""
    n, box = w.n_coarse, w.box
    e = np.zeros((n, n, n))
    e[tuple(cell)] = 1.0
    g = I.gradient_5pt(e, box / n)
    base4 = np.concatenate([e[..., None], np.moveaxis(g, 0, -1)], axis=-1)
    wts = np.asarray(w.slice_weight, dtype=np.float64)
    out = []
    # coarse level: the cells the 5-point stencil reaches
    ii, jj, kk = np.nonzero(np.abs(base4).sum(axis=-1) > 0)
    keys = I.morton3(ii, jj, kk)
    rows = np.searchsorted(w.levels[0].keys, keys)
    out.append((rows, base4[ii, jj, kk][:, None, :] * wts[None, :, None]))
    dx0 = box / n
    cc = (np.asarray(cell, dtype=np.float64) + 0.5) * dx0
    for lev in range(1, len(w.levels)):
        keys = w.levels[lev].keys
        ci, cj, ck = I._demorton(keys)
        xc = (np.stack([ci, cj, ck]).astype(np.float64) + 0.5) * (box / (n << lev))
        q = (xc - cc[:, None] + 0.5 * box) % box - 0.5 * box
        near = np.nonzero(np.abs(q).max(axis=0) < 4.0 * dx0)[0]
        rec = I.trilinear_periodic(base4, xc[:, near] / dx0)
        out.append((near, rec[:, None, :] * wts[None, :, None]))
    return out


def test_pullback_matches_oracle_differences_on_64_coarse_cells():
    """dL/dphi_0 for L = sum |xi - xi_FLRW|^2 on the differentiation workload's 64 x 64 patch
    against central differences of the oracle's loss, one coarse cell at a time (the oracle traces
    the rays that pass near the cell; the others are unchanged bit for bit)."""
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = _diff_patch()
    es = oracle.eta_stop(w.bg, float(w.z_max[0]))
    ref = w.observer[0][:, None] + w.dirs * (w.bg[-1, 0] - es)
    tree = _tree(w)
    p = B.TraceParams.from_workload(w)
    dirs_t = torch.from_numpy(w.dirs).cuda()
    base = B.trace_rays(tree, p, dirs_t)
    dxi = 2.0 * (base["xi"] - torch.from_numpy(ref).cuda())
    adj = B.trace_rays_adjoint(tree, p, dirs_t, jacobian=False, lensing=False, dL_dxi=dxi)
    g = B.pullback_coarse_phi(tree, adj["dL_drec"], w.slice_weight, w.n_coarse).cpu().numpy()
    torch.cuda.synchronize()
    tree.free()
    # 64 seeded cells among those within 2 cells of some ray's path (geometry only)
    rng = np.random.Generator(np.random.PCG64(4114))
    n = w.n_coarse
    picks = []
    while len(picks) < 64:
        cell = tuple(int(x) for x in rng.integers(0, n, size=3))
        if cell not in picks and _affected_rays(w, cell, 2.0).size:
            picks.append(cell)
    levels = [I.Level(l.keys, l.records.copy()) for l in w.levels]
    errs, kinked, detail = [], [], []
    gmax = np.abs(g).max()
    for cell in picks:
        rays = _affected_rays(w, cell, 5.5)
        wr = dataclasses.replace(w, dirs=np.ascontiguousarray(w.dirs[:, rays]),
                                 ray_begin=np.array([0, rays.size], dtype=np.int64))
        resp = _impulse_records(w, cell)
        fds, same = [], True
        for d in (1e-7, 5e-8):
            Ls, steps = [], []
            for sgn in (+1, -1):
                for l, (rows, r) in zip(levels, resp):
                    l.records[rows] += sgn * d * r
                o = oracle.trace(dataclasses.replace(wr, levels=levels))
                for l, l0, (rows, r) in zip(levels, w.levels, resp):
                    l.records[rows] = l0.records[rows]
                xi = oracle.xi_on_surface(o, es)
                Ls.append(float(((xi - ref[:, rays]) ** 2).sum()))
                steps.append(o["n_steps"])
            fds.append((Ls[0] - Ls[1]) / (2 * d))
            same = same and np.array_equal(steps[0], steps[1])
        rich = (4.0 * fds[1] - fds[0]) / 3.0
        m = int(I.morton3(np.array([cell[0]]), np.array([cell[1]]), np.array([cell[2]]))[0])
        gc = g[m]
        floor = 1e-4 * gmax
        # a kink of the piecewise-smooth loss between the two step sizes (a step count, a level or a
        # CIC cell plane crossed): the quotients disagree; reported, not judged
        if not same or abs(fds[0] - fds[1]) > 1e-5 * max(abs(rich), floor):
            kinked.append((cell, rays.size, fds, gc))
            continue
        errs.append(abs(rich - gc) / max(abs(rich), floor))
        detail.append((cell, rays.size, fds, gc))
    errs = np.array(errs)
    worst = int(np.argmax(errs))
    print("pull-back vs central differences: max", errs.max(), "median", np.median(errs), "judged", errs.size,
          "kinked", len(kinked), "worst", detail[worst], "gmax", gmax, "kinked picks", kinked)
    assert errs.size >= 56
    assert errs.max() < 1e-5, errs


def _rounded(w):
    """The workload with its records rounded to FP32 (held as FP64): the field an FP32 octree holds."""
    return dataclasses.replace(w, levels=[I.Level(l.keys, l.records.astype(np.float32).astype(np.float64))
                                          for l in w.levels])


def _vjp32(w, wxi, checkpoint_every=64):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, I.fp32_levels(w), w.bg, "fp32")
    r = B.trace_rays_adjoint(tree, B.TraceParams.from_workload(w), torch.from_numpy(w.dirs).cuda(), jacobian=False,
                             lensing=False, dL_dxi=torch.from_numpy(np.ascontiguousarray(wxi)).cuda(),
                             checkpoint_every=checkpoint_every)
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return [g.cpu().numpy() for g in r["dL_drec"]], r["status"].cpu().numpy()


@pytest.mark.parametrize("which", ["small", "diff_patch"])
def test_mixed_reverse_matches_the_fp64_derivative(which):
    """FP32 octree: the reverse sweep of the mixed-precision step (FP32 stages, FP64 state) applies
    the transpose of the same derivative as the FP64 form on the same FP32-rounded records, up to the
    mixed path's own rounding (its trajectories differ from FP64 by < 1e-4 relative): <v, J^T w>
    against <J v, w> of the FP64 forward derivative, and the record gradients level by level."""
    w = _rounded(_small() if which == "small" else _diff_patch())
    v = _direction(w, 31)
    wxi = np.random.Generator(np.random.PCG64(32)).normal(size=(3, w.n_rays))
    jv = _jvp(w, v)["dxi"]
    g32, st32 = _vjp32(w, wxi)
    g64, st64 = _vjp(w, wxi)
    assert (st32 == 0).all() and (st64 == 0).all()
    lhs = float((jv * wxi).sum())
    rhs = float(sum((a * b).sum() for a, b in zip(v, g32)))
    rel = abs(lhs - rhs) / abs(lhs)
    print(f"<J v, w> (FP64) {lhs:.12e}, <v, J^T w> (mixed) {rhs:.12e}, relative difference {rel:.2e}")
    assert rel < 1e-4
    for lev, (a, b) in enumerate(zip(g32, g64)):
        d = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"level {lev}: |g_mixed - g_fp64| / |g_fp64| = {d:.2e}")
        assert d < 1e-3


def test_mixed_reverse_checkpoint_interval_does_not_change_gradients():
    w = _small()
    wxi = np.random.Generator(np.random.PCG64(33)).normal(size=(3, w.n_rays))
    a, _ = _vjp32(w, wxi, 64)
    b, _ = _vjp32(w, wxi, 5)
    for x, y in zip(a, b):
        # same arithmetic in every segment layout; only the FP64 atomics' order differs
        np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("which", ["small", "diff_patch"])
def test_mixed_reverse_traces_the_same_map_as_the_forward_trace(which):
    """FP32 octree: the reverse mode differentiates the map mt_trace_rays computes, so the rays its
    forward pass and segment recomputes integrate are the trace's, bit for bit: every end-point
    output of mt_trace_rays_adjoint (record gradients requested) equals mt_trace_rays's."""
    import torch
    from paper_2111_08744_gb300 import binding as B
    w = _small() if which == "small" else _diff_patch()
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, I.fp32_levels(w), w.bg, "fp32")
    params = B.TraceParams.from_workload(w)
    dirs = torch.from_numpy(w.dirs).cuda()
    ref = B.trace_rays(tree, params, dirs)
    wxi = torch.from_numpy(np.random.Generator(np.random.PCG64(34)).normal(size=(3, w.n_rays))).cuda()
    got = B.trace_rays_adjoint(tree, params, dirs, jacobian=False, lensing=False, dL_dxi=wxi, checkpoint_every=16)
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    for k in B.OUT_F64 + B.OUT_I32 + ["xi"]:
        assert torch.equal(got[k], ref[k]), k


def test_field_model_forward_on_the_gpu_matches_the_generator():
    """mt_field_from_coarse_phi (phi_0 -> records of every level) against the generator's field model
    (inputs.records_from_phi0) for a random phi_0, element by element; it is the transpose of the
    pull-back: <records(v), rbar> - <records(0), rbar> = <v, pullback(rbar)>."""
    import torch
    from paper_2111_08744_gb300 import autograd as AG
    from paper_2111_08744_gb300 import binding as B
    w = _small()
    rng = np.random.Generator(np.random.PCG64(61))
    phi = rng.normal(size=(w.n_coarse,) * 3) * 1e-5
    tc = AG.TraceContext(w)
    got = [r.cpu().numpy() for r in tc.field_records(torch.from_numpy(phi).cuda())]
    ref = I.records_from_phi0(w, phi)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r.records, rtol=1e-12, atol=1e-12 * np.abs(r.records).max())
    # adjointness with the pull-back on the linear part
    rbar = [rng.normal(size=l.records.shape) for l in w.levels]
    key = tc.morton_index().cpu().numpy()
    v_m = np.empty(key.size)
    v_m[key] = phi.ravel()
    lin = [g - b.cpu().numpy() for g, b in zip(got, tc._base)]
    lhs = sum((a * b).sum() for a, b in zip(lin, rbar))
    tree = tc._geom
    pb = B.pullback_coarse_phi(tree, [torch.from_numpy(x).cuda() for x in rbar], w.slice_weight, w.n_coarse)
    rhs = float((pb.cpu().numpy() * v_m).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
