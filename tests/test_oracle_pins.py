"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form,
an invariant of the geodesic equations (Eqs. 1-3), brute force on a tiny tree,
or a statement the paper makes about its own method.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- background (Sect. 2.2 tables)

def test_background_matches_independent_quadrature():
    """eta(a) = int_{z(a)}^inf dz / H(z) (redshift-space quadrature, independent of the generator)."""
    bg = I.background_table(0.31)
    om, ol = 0.31, 0.69
    hz = lambda z: I.H0 * math.sqrt(om * (1 + z) ** 3 + ol)
    for ai, ei in zip(bg[::257, 1], bg[::257, 0]):
        z = 1.0 / ai - 1.0
        ref = quad(lambda t: 1.0 / hz(t), z, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]
        assert abs(ei - ref) < 1e-9 * ref
        assert abs(I.conformal_hubble(ai, om) - ai * hz(z)) < 1e-15


def test_background_interpolant_einstein_de_sitter_closed_form():
    # Om = 1: a = (H0 eta / 2)^2 and a'/a = 2 / eta exactly.
    bg = I.background_table(1.0)
    rng = np.random.Generator(np.random.PCG64(1))
    eta = rng.uniform(bg[0, 0], bg[-1, 0], 500)
    a, Hc = oracle.background(bg, eta)
    np.testing.assert_allclose(a, (I.H0 * eta / 2) ** 2, rtol=1e-12)
    np.testing.assert_allclose(Hc, 2.0 / eta, rtol=1e-12)


def test_eta_stop_inverts_background():
    bg = I.background_table(0.31)
    for z in (0.0, 0.3, 0.5, 1.0, 2.0):
        e = oracle.eta_stop(bg, z)
        a, _ = oracle.background(bg, e)
        assert abs(a[0] - 1.0 / (1.0 + z)) < 1e-14
    # comoving distance to z = 1 for Om = 0.31 (independent quadrature of dz/H)
    chi = quad(lambda z: 1.0 / (I.H0 * math.sqrt(0.31 * (1 + z) ** 3 + 0.69)), 0, 1.0, epsrel=1e-13)[0]
    assert abs((bg[-1, 0] - oracle.eta_stop(bg, 1.0)) - chi) < 1e-8 * chi


# ---------------------------------------------------------------- HEALPix inputs (Sect. 2.4)

def test_healpix_ring_nested_same_centres_and_counts():
    g = _golden("paper_values.json")
    for ns in (1, 2, 8, 16):
        npix = g["healpix_npix_factor"] * ns * ns
        d_r = I.healpix_directions(ns, nest=False)
        d_n = I.healpix_directions(ns, nest=True)
        assert d_r.shape[1] == npix == d_n.shape[1]
        a = {tuple(v) for v in np.round(d_r.T, 10)}
        b = {tuple(v) for v in np.round(d_n.T, 10)}
        assert a == b
        assert np.abs(d_r.sum(axis=1)).max() < 1e-9 * npix
        # ring latitudes: polar z = 1 - i^2/(3N^2), equatorial z = 4/3 - 2i/(3N)
        zs = np.unique(np.round(d_r[2], 12))
        ref = [1 - i * i / (3.0 * ns * ns) for i in range(1, ns)]
        ref += [4.0 / 3 - 2.0 * i / (3.0 * ns) for i in range(ns, 3 * ns + 1)]
        ref += [-(1 - i * i / (3.0 * ns * ns)) for i in range(1, ns)]
        np.testing.assert_allclose(np.sort(zs), np.sort(np.round(ref, 12)), atol=1e-11)


# ---------------------------------------------------------------- lookup and CIC (Sect. 2.2, Eq. 8, Fig. 1)

def _brute_levels(levels, n, box, pts, periodic=True):
    """Finest containing level and the level CIC uses, by scanning Python sets of (i, j, k)."""
    sets = []
    for lev, L in enumerate(levels):
        ci, cj, ck = I._demorton(L.keys)
        sets.append(set(zip(ci.tolist(), cj.tolist(), ck.tolist())))
    fin, cic = [], []
    for p in pts.T:
        u = p / (box / n)
        best = -1
        for lev in range(len(levels)):
            nl = n << lev
            c = tuple(int(math.floor(v * (1 << lev))) % nl for v in u)
            if c in sets[lev]:
                best = lev
            else:
                break
        fin.append(best)
        used = -1
        for lev in range(best, -1, -1):
            nl = n << lev
            i0 = [int(math.floor(v * (1 << lev) - 0.5)) for v in u]
            ok = all(((i0[0] + a) % nl, (i0[1] + b) % nl, (i0[2] + c) % nl) in sets[lev]
                     for a in (0, 1) for b in (0, 1) for c in (0, 1))
            if ok:
                used = lev
                break
        cic.append(used)
    return np.array(fin), np.array(cic)


def _brute_cic_value(level, lev, n, box, p):
    """Sum over EVERY cell of the level (and its periodic images) of W_CIC weights, Eq. (8)."""
    nl = n << lev
    dx = box / nl
    ci, cj, ck = I._demorton(level.keys)
    tot = np.zeros(4)
    wsum = 0.0
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                cx = (ci + 0.5 + sx * nl) * dx
                cy = (cj + 0.5 + sy * nl) * dx
                cz = (ck + 0.5 + sz * nl) * dx
                r = np.abs(np.stack([cx - p[0], cy - p[1], cz - p[2]])) / dx
                w = np.prod(np.clip(1.0 - r, 0.0, None), axis=0)
                tot += w @ level.records[:, 0, :]
                wsum += w.sum()
    return tot, wsum


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_lookup_and_fallback_match_brute_force(seed):
    n, box = 4, 40.0
    rng = np.random.Generator(np.random.PCG64(seed))
    fn = lambda xc: np.stack([np.sin(xc[0] / 7.0) + xc[1] * 0.01, np.cos(xc[1] / 5.0), xc[2] * 0.1, xc[0] * 0.02]).T
    levels = H.random_tree(n, 3, box, fn, seed, frac=0.4)
    pts = rng.uniform(0, box, size=(3, 400))
    w = H.workload(levels, box, n, I.healpix_directions(1))
    phi, grad, pe, lf, lc = oracle.sample(w, pts, w.bg[-1, 0])
    bf, bc = _brute_levels(levels, n, box, pts)
    np.testing.assert_array_equal(lf, bf)
    np.testing.assert_array_equal(lc, bc)
    # interpolated value equals the all-cells W_CIC sum at the chosen level
    for i in range(0, 400, 23):
        tot, wsum = _brute_cic_value(levels[lc[i]], lc[i], n, box, pts[:, i])
        assert abs(wsum - 1.0) < 1e-12
        np.testing.assert_allclose([phi[i], *grad[:, i]], tot, rtol=1e-12, atol=1e-14)


def test_fig1_fallback_cases():
    """The four situations of Fig. 1 (2D there, 3D here) on a hand-built tree."""
    n, box = 4, 4.0
    fn = H.const_fn(0.0)
    l0 = H.coarse_level_from_fn(n, box, fn)
    # refine coarse cells x in {1, 2}, y in {1, 2}, z in {1, 2} (a 2^3 block) and one isolated cell (0, 3, 3)
    par = [I.morton3(i, j, k) for i in (1, 2) for j in (1, 2) for k in (1, 2)] + [I.morton3(0, 3, 3)]
    l1 = H.refined_level_from_parents(np.array(par, dtype=np.uint64), 1, n, box, fn)
    w = H.workload([l0, l1], box, n, I.healpix_directions(1))
    pts = np.array([
        [0.5, 0.5, 0.5],      # coarse-only region: finest 0, CIC 0
        [2.0, 2.0, 2.0],      # centre of the refined block: finest 1, CIC 1
        [1.1, 1.1, 1.1],      # refined cell at the block's edge, fine neighbours missing: finest 1, CIC 0
        [0.9, 3.6, 3.6],      # isolated refined octet, off its central quarter: a fine neighbour is missing
        [0.5, 3.5, 3.5],      # the octet's centre: its 8 fine cells are the CIC neighbours
    ]).T
    _, _, _, lf, lc = oracle.sample(w, pts, w.bg[-1, 0])
    np.testing.assert_array_equal(lf, [0, 1, 1, 1, 1])
    np.testing.assert_array_equal(lc, [0, 1, 0, 0, 1])


def test_cic_reproduces_linear_fields_and_partition_of_unity():
    n, box = 8, 80.0
    g = np.array([1e-6, -2e-6, 3e-6])
    levels = H.random_tree(n, 2, box, H.linear_fn(g, 1e-5), seed=11, frac=0.5)
    w = H.workload(levels, box, n, I.healpix_directions(1), periodic=0)
    rng = np.random.Generator(np.random.PCG64(7))
    pts = rng.uniform(box / n, box - box / n, size=(3, 300))   # away from the non-periodic edge
    phi, grad, pe, lf, lc = oracle.sample(w, pts, w.bg[-1, 0])
    assert (lc >= 0).all()
    np.testing.assert_allclose(phi, 1e-5 + g @ pts, rtol=0, atol=1e-17 * box * 10 + 1e-18)
    np.testing.assert_allclose(grad, np.repeat(g[:, None], pts.shape[1], axis=1), rtol=1e-13)
    ones = H.random_tree(n, 2, box, H.const_fn(1.0), seed=11, frac=0.5)
    w1 = H.workload(ones, box, n, I.healpix_directions(1))
    phi1, *_ = oracle.sample(w1, rng.uniform(0, box, size=(3, 300)), w.bg[-1, 0])
    np.testing.assert_allclose(phi1, 1.0, rtol=1e-14)


def test_time_slices_linear_in_eta():
    n, box = 4, 40.0
    bg = I.background_table(0.31)
    seta = np.array([oracle.eta_stop(bg, 1.0), bg[-1, 0]])
    lv = [H.coarse_level_from_fn(n, box, H.const_fn(1e-5), n_slices=2, slice_scale=[1.3, 1.0])]
    w = H.workload(lv, box, n, I.healpix_directions(1), slice_eta=seta)
    for e, ref in ((seta[0], 1.3e-5), (seta[1], 1e-5), (0.5 * (seta[0] + seta[1]), 1.15e-5)):
        phi, grad, pe, *_ = oracle.sample(w, np.array([[3.0], [5.0], [7.0]]), e)
        assert abs(phi[0] - ref) < 1e-18
        assert abs(pe[0] - (1e-5 - 1.3e-5) / (seta[1] - seta[0])) < 1e-22


# ---------------------------------------------------------------- geodesics (Eqs. 1-4, 23-28)

def test_flrw_rays_are_straight_and_redshift_exact():
    """phi = 0: straight rays, eta_o - eta = chi, k0 a^2 = -1, z5 = z0 (Sect. 3.4: FLRW redshift
    recovered to double precision with RK4 at 4 steps per cell)."""
    w = I.config_plain_small()
    w.steps_per_cell = 4
    o = oracle.trace(w, gravity_on=False)
    assert (o["status"] == 0).all()
    d = o["x"] - w.observer[0][:, None]
    chi = o["chi"]
    trans = d - (d * w.dirs).sum(0) * w.dirs
    assert np.abs(trans).max() < 1e-10 * chi.max()
    np.testing.assert_allclose(w.bg[-1, 0] - o["eta"], chi, rtol=1e-13)
    a_s, _ = oracle.background(w.bg, o["eta"])
    np.testing.assert_allclose(np.abs(o["k"][0]) * a_s * a_s, 1.0, rtol=1e-12)
    np.testing.assert_allclose(o["z5"], o["z0"], rtol=1e-12)
    np.testing.assert_allclose(o["path"], chi, rtol=1e-13)
    assert np.abs(o["z0"] - 0.5).max() < 1e-6
    # without AMR the step count is n_steps * chi / x_coarse (Sect. 3.1, after Eq. 29)
    steps = w.steps_per_cell * chi / (w.box / w.n_coarse)
    assert np.abs(o["n_steps"] - steps).max() <= 1.0


def test_constant_gradient_gives_analytic_deflection():
    """phi = g.x: to first order d^2 x_perp / d chi^2 = -2 grad_perp phi, so x_perp = -g_perp chi^2."""
    n, box = 16, 4000.0
    g = np.array([2e-9, -1e-9, 1.5e-9])
    lv = [H.coarse_level_from_fn(n, box, H.linear_fn(g, 0.0))]
    dirs = I.healpix_directions(2)
    w = H.workload(lv, box, n, dirs, z_max=0.4, periodic=0, steps_per_cell=8)
    o = oracle.trace(w)
    assert (o["status"] == 0).all()
    x0 = w.observer[0][:, None]
    d = o["x"] - x0
    along = (d * dirs).sum(0)
    trans = d - along * dirs
    gperp = g[:, None] - (g[:, None] * dirs).sum(0) * dirs
    ref = -gperp * along ** 2
    err = np.abs(trans - ref).max() / np.abs(ref).max()
    assert err < 5e-3, err


def test_null_condition_and_redshift_consistency_on_linear_field():
    """Where the interpolated gradient is the gradient of the interpolated potential (a linear
    field, which CIC reproduces exactly), the null condition of Eq. (1),
    -(1+2phi) k0^2 + (1-2phi)|k|^2 = 0, holds to first order along the ray, and z5 (Eq. 28)
    agrees with the decomposition z4 (Eq. 27) to second order in phi."""
    n, box = 16, 4000.0
    g = np.array([3e-9, 1e-9, -2e-9])
    lv = [H.coarse_level_from_fn(n, box, H.linear_fn(g, 2e-6))]
    # 32 steps per 250 h^-1 Mpc cell keeps the RK4 truncation error (~h^4) below phi^2
    w = H.workload(lv, box, n, I.healpix_directions(2), z_max=0.45, periodic=0, steps_per_cell=32)
    o = oracle.trace(w)
    assert (o["status"] == 0).all()
    k0 = o["k"][0]
    kk = (o["k"][1:] ** 2).sum(0)
    C = -(1 + 2 * o["phi_s"]) * k0 ** 2 + (1 - 2 * o["phi_s"]) * kk
    # second order: phi^2 ~ 1e-10 here; a wrong sign of a first-order term would give ~4 phi ~ 3e-5
    assert np.abs(C / k0 ** 2).max() < 5e-9
    assert np.abs(o["z5"] - o["z4"]).max() < 5e-9
    assert np.abs(o["z5"] - o["z0"]).max() > 1e-6


def test_grf_gravity_is_small_and_consistent():
    """On the k^-3 random field the potential and force records are interpolated separately
    (Sect. 2.2), so the null condition drifts only at the level of their grid-scale mismatch."""
    w = I.config_plain_small()
    o = oracle.trace(w)
    k0 = o["k"][0]
    C = -(1 + 2 * o["phi_s"]) * k0 ** 2 + (1 - 2 * o["phi_s"]) * (o["k"][1:] ** 2).sum(0)
    assert np.abs(C / k0 ** 2).max() < 1e-3
    assert 1e-6 < np.abs(o["z5"] - o["z0"]).max() < 1e-3
    assert np.abs(o["z1"] - o["z0"]).max() < 1e-4


def test_uniform_time_varying_potential_isw():
    """phi(eta) uniform in space and linear in eta: I = phi_o - phi_s exactly, k0 follows FLRW,
    and z5 = z4 = z0 - (phi_o - phi_s)/a to first order (Eqs. 24, 27, 28)."""
    n, box = 8, 1000.0
    bg = I.background_table(0.31)
    seta = np.array([oracle.eta_stop(bg, 1.0), bg[-1, 0]])
    lv = [H.coarse_level_from_fn(n, box, H.const_fn(1e-5), n_slices=2, slice_scale=[2.0, 1.0])]
    w = H.workload(lv, box, n, I.healpix_directions(1), z_max=0.8, slice_eta=seta, steps_per_cell=64)
    o = oracle.trace(w)
    np.testing.assert_allclose(o["isw"], o["phi_o"] - o["phi_s"], rtol=1e-10)
    a_s, _ = oracle.background(bg, o["eta"])
    np.testing.assert_allclose(np.abs(o["k"][0]) * a_s ** 2, 1.0, rtol=1e-11)
    ref = o["z0"] - (o["phi_o"] - o["phi_s"]) / a_s
    np.testing.assert_allclose(o["z4"], ref, rtol=0, atol=1e-15)
    assert np.abs(o["z5"] - o["z4"]).max() < 1e-9
    assert np.abs(o["z4"] - o["z0"]).max() > 1e-6


def test_rk4_fourth_order_on_flrw():
    """Step halving on an FLRW ray with coarse cells: the k0 error against the analytic k0 a^2 = -1
    falls by ~2^4 per halving (classical RK4, Sect. 2.2)."""
    n, box = 4, 1000.0
    lv = [H.coarse_level_from_fn(n, box, H.const_fn(0.0))]
    errs = []
    for N in (1, 2, 4):
        w = H.workload(lv, box, n, I.healpix_directions(1)[:, :1], z_max=2.0, steps_per_cell=N)
        o = oracle.trace(w, gravity_on=False)
        a_s, _ = oracle.background(w.bg, o["eta"])
        errs.append(abs(abs(o["k"][0][0]) * a_s[0] ** 2 - 1.0))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, errs


def test_rk4_fourth_order_with_the_gravitational_terms():
    """Step halving through the smooth analytic potential phi = A sin(k . x) (exact phi and grad phi,
    no interpolation kinks): the error of the gravitational displacement of the end point (the
    difference from the same ray without gravity, so that the background's own error cancels)
    against a 512-steps-per-cell reference falls by ~2^4 per halving (RK4 of Eqs. 2-4, Sect. 2.2)."""
    n, box = 4, 1000.0
    lv = [H.coarse_level_from_fn(n, box, H.const_fn(0.0))]
    k = 2.0 * np.pi / box * np.array([3.0, 2.0, 1.0])
    an = np.array([3e-4, *k])
    dirs = I.healpix_directions(2)[:, [3, 17, 30]]

    def displacement(N):
        w = H.workload(lv, box, n, dirs, z_max=1.0, steps_per_cell=N)
        es = oracle.eta_stop(w.bg, 1.0)
        g = oracle.trace(w, analytic=an)
        f = oracle.trace(w, gravity_on=False)
        return oracle.xi_on_surface(g, es) - oracle.xi_on_surface(f, es)

    ref = displacement(512)
    assert np.abs(ref).max() > 0.1     # a deflection of order 1 h^-1 Mpc
    errs = [np.abs(displacement(N) - ref).max() for N in (4, 8, 16, 32)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(13 < r < 21 for r in ratios), (errs, ratios)


def quadratic_fn(Q, x0):
    """phi = (x - x0)^T Q (x - x0) / 2 with records of its exact (linear) gradient Q (x - x0)."""
    Q = np.asarray(Q, dtype=np.float64)

    def fn(xc):
        d = xc - np.asarray(x0, dtype=np.float64)[:, None]
        rec = np.empty((xc.shape[1], 4))
        rec[:, 0] = 0.5 * np.einsum("in,ij,jn->n", d, Q, d)
        rec[:, 1:] = (Q @ d).T
        return rec

    return fn


def test_finite_beam_identity_without_gravity():
    w = I.config_plain_small()
    dirs = w.dirs[:, ::97]
    A0 = oracle.bundle_jacobian(w, dirs=dirs, eps=1e-6, gravity_on=False)
    np.testing.assert_allclose(A0[[0, 3]], 1.0, atol=1e-8)
    np.testing.assert_allclose(A0[[1, 2]], 0.0, atol=1e-8)


def test_finite_beam_matches_born_closed_form_for_quadratic_potential():
    """phi = x^T Q x / 2 (constant Hessian, curl-free linear force reproduced exactly by CIC):
    Eq. (12) gives A = I - 2 Q_perp int_0^chi (chi - c) c / chi dc = I - (chi^2 / 3) Q_perp on the
    screen (e1, e2).  The finite beam of Eq. (21) must agree to first order."""
    n, box = 16, 4000.0
    xo = np.array([2000.0, 2000.0, 2000.0])
    Q = np.array([[4e-10, 1e-10, 0.0], [1e-10, -2e-10, 0.5e-10], [0.0, 0.5e-10, 1e-10]])
    lv = [H.coarse_level_from_fn(n, box, quadratic_fn(Q, xo))]
    dirs = I.healpix_directions(2)
    w = H.workload(lv, box, n, dirs, z_max=0.45, periodic=0, steps_per_cell=8, observer=xo)
    A = oracle.bundle_jacobian(w, eps=1e-5)
    o = oracle.trace(w)
    chi = o["chi"]

    def screen(v):
        v = v / np.linalg.norm(v, axis=0)
        t1, t2 = np.arctan2(v[1], v[0]), np.arccos(v[2])
        return [np.stack([-np.sin(t1), np.cos(t1), np.zeros_like(t1)]),
                np.stack([-np.cos(t1) * np.cos(t2), -np.sin(t1) * np.cos(t2), np.sin(t2)])]

    E = screen(dirs)                                            # e1, e2 at the observed direction
    xi = oracle.xi_on_surface(o, oracle.eta_stop(w.bg, 0.45))
    Et = screen(xi - xo[:, None])                               # beta-screen at the source direction
    qnn = np.einsum("in,ij,jn->n", dirs, Q, dirs)
    scale = chi.max() ** 2 / 3.0 * np.abs(Q).max()
    for a in range(2):
        for b in range(2):
            # angular Hessian of phi on the sphere: chi^2 (Q_ab - Q_nn delta_ab); the beta-screen basis
            # differs from the observer's by M_ab = e~_a(beta) . e_b(theta) (first order in deflection)
            M = (Et[a] * E[b]).sum(0)
            qab = np.einsum("in,ij,jn->n", E[a], Q, E[b]) - (qnn if a == b else 0.0)
            ref = M - chi ** 2 / 3.0 * qab
            dev = np.abs(A[2 * a + b] - ref)
            assert dev.max() < 0.01 * scale, (a, b, dev.max(), scale)


def test_fp32_field_changes_results_only_slightly():
    w = I.config_plain_small()
    sub = w.dirs[:, ::31]
    o64 = oracle.trace(w, dirs=sub)
    o32 = oracle.trace(w, dirs=sub, levels=I.fp32_levels(w))
    np.testing.assert_allclose(o32["x"], o64["x"], rtol=1e-9, atol=1e-6)


def test_step_size_follows_refinement_level():
    """N steps per AMR cell (Sect. 2.2): a tree refined everywhere to level 2 takes 4x the steps of
    its coarse grid along the same FLRW ray."""
    n, box = 8, 1000.0
    fn = H.const_fn(0.0)
    l0 = H.coarse_level_from_fn(n, box, fn)
    l1 = H.refined_level_from_parents(l0.keys, 1, n, box, fn)
    l2 = H.refined_level_from_parents(l1.keys, 2, n, box, fn)
    dirs = I.healpix_directions(1)
    w0 = H.workload([l0], box, n, dirs, z_max=0.3)
    w2 = H.workload([l0, l1, l2], box, n, dirs, z_max=0.3)
    o0 = oracle.trace(w0, gravity_on=False)
    o2 = oracle.trace(w2, gravity_on=False)
    assert (o2["level"] == 2).all() and (o0["level"] == 0).all()
    chi = o0["chi"]
    assert np.abs(o0["n_steps"] - 4 * chi / (box / n)).max() <= 1
    assert np.abs(o2["n_steps"] - 16 * chi / (box / n)).max() <= 1
    # the end points, moved onto the iso-eta surface, agree (FLRW: straight rays)
    es = oracle.eta_stop(w0.bg, 0.3)
    d0 = np.linalg.norm(oracle.xi_on_surface(o0, es) - w0.observer[0][:, None], axis=0)
    d2 = np.linalg.norm(oracle.xi_on_surface(o2, es) - w0.observer[0][:, None], axis=0)
    np.testing.assert_allclose(d2, d0, rtol=1e-11)


# ---------------------------------------------------------------- iso-chi stop (Sect. 2.5 geodesic finder)

def test_iso_chi_stop_flrw_and_constant_gradient():
    """FLRW: the ray ends exactly on the sphere along its direction; phi = g.x: the end point on
    the sphere |x - x_o| = chi is deflected by x_perp = -g_perp chi^2 (first order)."""
    n, box = 16, 4000.0
    g = np.array([2e-9, -1e-9, 1.5e-9])
    lv = [H.coarse_level_from_fn(n, box, H.linear_fn(g, 0.0))]
    dirs = I.healpix_directions(2)
    w = H.workload(lv, box, n, dirs, z_max=0.4, periodic=0, steps_per_cell=8)
    chi = np.linspace(300.0, 1400.0, dirs.shape[1])
    x0 = w.observer[0][:, None]
    flrw = oracle.trace(w, gravity_on=False, chi_stop=chi)
    assert (flrw["status"] == 0).all()
    np.testing.assert_allclose(flrw["x"], x0 + chi * dirs, rtol=0, atol=1e-9)
    o = oracle.trace(w, chi_stop=chi)
    d = o["x"] - x0
    np.testing.assert_allclose(np.linalg.norm(d, axis=0), chi, rtol=1e-12)
    along = (d * dirs).sum(0)
    trans = d - along * dirs
    gperp = g[:, None] - (g[:, None] * dirs).sum(0) * dirs
    ref = -gperp * along ** 2
    assert np.abs(trans - ref).max() / np.abs(ref).max() < 5e-3
    # eta at the sphere: eta_o - chi in FLRW
    np.testing.assert_allclose(flrw["eta"], w.bg[-1, 0] - chi, rtol=0, atol=1e-8)
