"""Geodesic finder on the GPU (mt_find_geodesics, Sect. 2.5, Eq. 22), checked against its defining
equation with the oracle: the oracle traces each found direction to the source's sphere (its own
iso-chi stop) and must see the source in its direction."""
import functools

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def amr_small():
    return I.config_amr(n=64, box=500.0, n_levels=2, f1=0.04, ratio=0.3, nside=8, z_max=0.5, seed=31,
                        name="amr_64cube_L2_nside8")


def _sources(w, n, seed, chi_lo=100.0, chi_hi=1000.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=(3, n))
    v /= np.linalg.norm(v, axis=0)
    chi = rng.uniform(chi_lo, chi_hi, n)
    return w.observer[0][:, None] + chi * v, chi, v


def _find(w, precision, src, tol, gravity_on=True, interp="cic", max_newton=10, max_grid=20):
    import torch
    from paper_2111_08744_gb300 import binding as B
    tree = B.Octree(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, precision)
    cap = B.step_cap(w.bg, w.box / w.n_coarse, len(w.levels) - 1, w.steps_per_cell, 3.0)
    p = B.TraceParams(w.observer, [0.0], [0, src.shape[1]], w.steps_per_cell, gravity_on, cap, interp)
    r = B.find_geodesics(tree, p, torch.from_numpy(np.ascontiguousarray(src)).cuda(), tol=tol, max_newton=max_newton,
                         max_grid=max_grid)
    torch.cuda.synchronize()
    assert tree.device_status() == B.MT_OK
    tree.free()
    return {k: v.cpu().numpy() for k, v in r.items()}


def _oracle_beta(w, theta, chi, gravity_on=True, interp="cic"):
    o = oracle.trace(w, dirs=np.ascontiguousarray(theta), chi_stop=chi, gravity_on=gravity_on, interp=interp)
    d = o["x"] - w.observer[0][:, None]
    return d / np.linalg.norm(d, axis=0), o


def test_without_gravity_theta_is_beta():
    w = amr_small()
    src, chi, v = _sources(w, 64, 1)
    r = _find(w, "fp64", src, 1e-12, gravity_on=False)
    assert (r["fstatus"] == 0).all()
    np.testing.assert_allclose(r["theta"], v, atol=1e-12)
    assert (r["iters"] == 1).all()


@pytest.mark.parametrize("interp", ["cic", "tsc"])
def test_fp64_solutions_satisfy_the_lens_equation(interp):
    w = amr_small()
    src, chi, v = _sources(w, 256, 2)
    r = _find(w, "fp64", src, 1e-11, interp=interp)
    st = r["fstatus"]
    print("status counts", np.bincount(st, minlength=4), "iters max", r["iters"].max())
    assert np.mean(st <= 1) >= 0.98
    ok = st <= 1
    beta, o = _oracle_beta(w, r["theta"][:, ok], chi[ok], interp=interp)
    err = np.linalg.norm(beta - v[:, ok], axis=0)
    print("oracle |beta - beta_src|: max", err.max(), "deflection median",
          np.median(np.linalg.norm(r["theta"][:, ok] - v[:, ok], axis=0)))
    assert err.max() < 1e-9
    # the photon really was deflected (the solve did something)
    assert np.median(np.linalg.norm(r["theta"] - v, axis=0)) > 1e-7
    # the solution ray's outputs are those of that ray at the sphere
    np.testing.assert_allclose(r["x"][:, ok], o["x"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(r["z5"][ok], o["z5"], rtol=1e-9, atol=1e-12)


def test_fp32_field_mixed_solutions():
    w = amr_small()
    src, chi, v = _sources(w, 256, 3)
    r = _find(w, "fp32", src, 1e-10)
    ok = r["fstatus"] <= 1
    assert ok.mean() >= 0.97
    beta, _ = _oracle_beta(w, r["theta"][:, ok], chi[ok])
    err = np.linalg.norm(beta - v[:, ok], axis=0)
    print("mixed: oracle residual median", np.median(err), "max", err.max())
    assert np.median(err) < 1e-8 and np.mean(err < 1e-6) >= 0.97


def test_grid_fallback_reduces_the_residual():
    """One Newton iteration, then the shrinking grid: each round keeps the best of 25 directions, so
    the residual never grows and ends far below the first iterate's."""
    w = amr_small()
    src, chi, v = _sources(w, 64, 4)
    one = _find(w, "fp64", src, 1e-14, max_newton=1, max_grid=0)
    grid = _find(w, "fp64", src, 1e-14, max_newton=1, max_grid=12)
    assert (grid["fstatus"] != 3).all()
    assert (grid["resid"] <= one["resid"] * (1 + 1e-12)).all()
    assert np.median(grid["resid"]) < 0.05 * np.median(one["resid"])
    # traces: the Newton iterate, one per grid round (a source may converge and stop early), the final one
    assert (grid["iters"] <= 1 + 12 + 1).all()
    assert ((grid["iters"] == 1 + 12 + 1) | (grid["fstatus"] == 1)).all()
    beta, _ = _oracle_beta(w, grid["theta"], chi)
    # the oracle's map and the GPU's FP64 map differ by ~1e-11 rad
    np.testing.assert_allclose(np.linalg.norm(beta - v, axis=0), grid["resid"], rtol=1e-3, atol=3e-11)
