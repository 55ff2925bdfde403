"""Pins of the oracle's NGP (Eq. 7) and TSC (Eq. 9) interpolation with the level fallback of
Sect. 2.2, against brute force over every cell of tiny trees, a closed form of the TSC kernel on
quadratic fields, the hand-worked fallback situations of the TSC figure, and the closed-form
trajectories that hold for any scheme reproducing linear forces."""
import math

import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests import helpers as H


def _w_tsc(r):
    """Eq. (9), written out again for the brute force (vectorised)."""
    a = np.abs(r)
    return np.where(a < 0.5, 0.75 - r * r, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def _cell_sets(levels):
    sets, rows = [], []
    for L in levels:
        ci, cj, ck = I._demorton(L.keys)
        t = list(zip(ci.tolist(), cj.tolist(), ck.tolist()))
        sets.append(set(t))
        rows.append({c: r for r, c in enumerate(t)})
    return sets, rows


def _brute(levels, n, box, pts):
    """Finest containing level, and the level TSC uses: the finest one at or below it where the
    containing cell and all 26 neighbours exist (periodic)."""
    sets, _ = _cell_sets(levels)
    fin, tsc = [], []
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
            c = [int(math.floor(v * (1 << lev))) for v in u]
            if all(((c[0] + a) % nl, (c[1] + b) % nl, (c[2] + d) % nl) in sets[lev]
                   for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)):
                used = lev
                break
        tsc.append(used)
    return np.array(fin), np.array(tsc)


def _brute_tsc_value(level, lev, n, box, p):
    """Sum over EVERY cell of the level (and its periodic images) of the W_TSC product weights."""
    nl = n << lev
    dx = box / nl
    ci, cj, ck = I._demorton(level.keys)
    tot, wsum = np.zeros(4), 0.0
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                r = np.stack([(ci + 0.5 + sx * nl) * dx - p[0], (cj + 0.5 + sy * nl) * dx - p[1],
                              (ck + 0.5 + sz * nl) * dx - p[2]]) / dx
                w = np.prod(_w_tsc(r), axis=0)
                tot += w @ level.records[:, 0, :]
                wsum += w.sum()
    return tot, wsum


def _fn(xc):
    return np.stack([np.sin(xc[0] / 7.0) + xc[1] * 0.01, np.cos(xc[1] / 5.0), xc[2] * 0.1, xc[0] * 0.02]).T


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_tsc_and_ngp_lookup_match_brute_force(seed):
    n, box = 4, 40.0
    rng = np.random.Generator(np.random.PCG64(seed))
    levels = H.random_tree(n, 3, box, _fn, seed, frac=0.9)
    pts = rng.uniform(0, box, size=(3, 400))
    w = H.workload(levels, box, n, I.healpix_directions(1))
    bf, bt = _brute(levels, n, box, pts)
    phi, grad, pe, lf, lt = oracle.sample(w, pts, w.bg[-1, 0], interp="tsc")
    np.testing.assert_array_equal(lf, bf)
    np.testing.assert_array_equal(lt, bt)
    assert len(set(lt.tolist())) >= 3            # the draw exercises the fallback
    for i in range(0, 400, 19):
        tot, wsum = _brute_tsc_value(levels[lt[i]], lt[i], n, box, pts[:, i])
        assert abs(wsum - 1.0) < 1e-12
        np.testing.assert_allclose([phi[i], *grad[:, i]], tot, rtol=1e-12, atol=1e-14)
    # NGP: the records of the most refined cell containing the point, no fallback
    _, rows = _cell_sets(levels)
    phn, grn, _, lfn, ln = oracle.sample(w, pts, w.bg[-1, 0], interp="ngp")
    np.testing.assert_array_equal(ln, bf)
    for i in range(pts.shape[1]):
        lev = bf[i]
        c = tuple(int(math.floor(v / (box / n) * (1 << lev))) % (n << lev) for v in pts[:, i])
        rec = levels[lev].records[rows[lev][c], 0]
        assert phn[i] == rec[0] and (grn[:, i] == rec[1:]).all()


def test_tsc_quadratic_closed_form():
    """For q(x) = x.Qx/2 + b.x + c sampled at cell centres, TSC returns q(x) + dx^2 tr(Q)/8 (its
    second moment is 1/4 per axis, its first moment 0) and the linear gradient exactly."""
    n, box = 16, 160.0
    dx = box / n
    Q = np.array([[2e-6, 0.5e-6, -0.3e-6], [0.5e-6, -1e-6, 0.2e-6], [-0.3e-6, 0.2e-6, 0.6e-6]])
    b = np.array([1e-5, -2e-5, 0.5e-5])

    def fn(xc):
        rec = np.empty((xc.shape[1], 4))
        rec[:, 0] = 0.5 * np.einsum("in,ij,jn->n", xc, Q, xc) + b @ xc + 3e-5
        rec[:, 1:] = (Q @ xc).T + b
        return rec

    w = H.workload([H.coarse_level_from_fn(n, box, fn)], box, n, I.healpix_directions(1), periodic=0)
    rng = np.random.Generator(np.random.PCG64(9))
    pts = rng.uniform(2 * dx, box - 2 * dx, size=(3, 300))
    phi, grad, _, _, lt = oracle.sample(w, pts, w.bg[-1, 0], interp="tsc")
    assert (lt == 0).all()
    q = 0.5 * np.einsum("in,ij,jn->n", pts, Q, pts) + b @ pts + 3e-5
    np.testing.assert_allclose(phi, q + dx * dx * np.trace(Q) / 8.0, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(grad, Q @ pts + b[:, None], rtol=1e-12, atol=1e-16)
    # CIC on the same field is not exact for the quadratic part (the pin separates the kernels)
    phc, *_ = oracle.sample(w, pts, w.bg[-1, 0], interp="cic")
    assert np.abs(phc - q - dx * dx * np.trace(Q) / 8.0).max() > 1e-8


def test_tsc_fallback_cases():
    """The situations of the TSC figure (2D there, 3D here) on a hand-built tree: the 27 cells
    depend only on the cell containing the photon, not on its position inside it."""
    n, box = 4, 4.0
    fn = H.const_fn(0.0)
    l0 = H.coarse_level_from_fn(n, box, fn)
    par = [I.morton3(i, j, k) for i in (1, 2) for j in (1, 2) for k in (1, 2)] + [I.morton3(0, 3, 3)]
    l1 = H.refined_level_from_parents(np.array(par, dtype=np.uint64), 1, n, box, fn)
    w = H.workload([l0, l1], box, n, I.healpix_directions(1))
    pts = np.array([
        [0.5, 0.5, 0.5],      # coarse only: TSC at level 0
        [2.0, 2.0, 2.0],      # fine cell (4,4,4): fine neighbours 3..5 all inside the block
        [1.6, 1.6, 1.6],      # fine cell (3,3,3): neighbours 2..4, inside the block
        [1.9, 1.9, 1.9],      # same fine cell, other position: same answer
        [1.1, 1.1, 1.1],      # fine cell (2,2,2): neighbour 1 lies in an unrefined coarse cell
        [0.5, 3.5, 3.5],      # isolated octet: its cells always lack neighbours
    ]).T
    _, _, _, lf, lt = oracle.sample(w, pts, w.bg[-1, 0], interp="tsc")
    np.testing.assert_array_equal(lf, [0, 1, 1, 1, 1, 1])
    np.testing.assert_array_equal(lt, [0, 1, 1, 1, 0, 0])
    # CIC at the block's inner corner (1.6 -> fine 3.2): its 8 neighbours exist too
    _, _, _, _, lc = oracle.sample(w, pts, w.bg[-1, 0], interp="cic")
    np.testing.assert_array_equal(lc[:4], [0, 1, 1, 1])


@pytest.mark.parametrize("interp", ["ngp", "tsc"])
def test_constant_gradient_deflection_any_scheme(interp):
    """NGP and TSC both return a constant force exactly: x_perp = -g_perp chi^2 as for CIC."""
    n, box = 16, 4000.0
    g = np.array([2e-9, -1e-9, 1.5e-9])
    lv = [H.coarse_level_from_fn(n, box, H.linear_fn(g, 0.0))]
    dirs = I.healpix_directions(2)
    w = H.workload(lv, box, n, dirs, z_max=0.4, periodic=0, steps_per_cell=8)
    o = oracle.trace(w, interp=interp)
    assert (o["status"] == 0).all()
    d = o["x"] - w.observer[0][:, None]
    along = (d * dirs).sum(0)
    trans = d - along * dirs
    gperp = g[:, None] - (g[:, None] * dirs).sum(0) * dirs
    ref = -gperp * along ** 2
    assert np.abs(trans - ref).max() / np.abs(ref).max() < 5e-3


def test_tsc_finite_beam_matches_quadratic_closed_form():
    """TSC reproduces the linear force of a quadratic potential: the finite-beam distortion matrix
    obeys A = M - (chi^2/3)(Q_ab - Q_nn delta_ab) as for CIC (first order, beta-screen rotation M)."""
    n, box = 16, 4000.0
    xo = np.array([2000.0, 2000.0, 2000.0])
    Q = np.array([[4e-10, 1e-10, 0.0], [1e-10, -2e-10, 0.5e-10], [0.0, 0.5e-10, 1e-10]])

    def fn(xc):
        d = xc - xo[:, None]
        rec = np.empty((xc.shape[1], 4))
        rec[:, 0] = 0.5 * np.einsum("in,ij,jn->n", d, Q, d)
        rec[:, 1:] = (Q @ d).T
        return rec

    dirs = I.healpix_directions(2)
    w = H.workload([H.coarse_level_from_fn(n, box, fn)], box, n, dirs, z_max=0.45, periodic=0, steps_per_cell=8,
                   observer=xo)
    A_t = oracle.bundle_jacobian(w, eps=1e-5, interp="tsc")
    A_c = oracle.bundle_jacobian(w, eps=1e-5, interp="cic")
    o = oracle.trace(w, interp="tsc")
    chi = o["chi"]
    scale = chi.max() ** 2 / 3.0 * np.abs(Q).max()
    # both schemes see the same linear force field (away from the edge), so the same matrix
    assert np.abs(A_t - A_c).max() < 1e-3 * scale
    assert np.abs(A_t - np.eye(2).reshape(4, 1)).max() > 0.1 * scale   # lensing present
