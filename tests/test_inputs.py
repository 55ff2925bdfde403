"""The seeded synthetic workloads follow their stated recipe (they stand in for the paper's RayGal and
DEUS-FUR light cones): Gaussian potential with rms exactly 1e-5 and a k^-3 spectrum, 4th-order
gradients, refinement of the densest cells in whole octets at the stated volume fractions, the
growth normalisation of the time slices, and the ray sets' geometry."""
import math

import numpy as np

from paper_2111_08744_gb300 import inputs as I


def test_gaussian_potential_rms_mean_and_spectrum():
    n, box = 64, 1000.0
    f = I.gaussian_potential(n, box, seed=5, rms=1e-5)
    assert abs(np.sqrt(np.mean(f * f)) - 1e-5) < 1e-17
    assert abs(f.mean()) < 1e-20
    # spherically averaged power: P(k) ~ k^-3 between the fundamental and the Nyquist range
    pk = np.abs(np.fft.rfftn(f)) ** 2
    kx, ky, kz = I._kgrid(n, box)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kf = 2 * math.pi / box
    edges = kf * np.geomspace(2, n / 4, 12)
    mids, pw = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (kk >= lo) & (kk < hi)
        mids.append(np.sqrt(lo * hi))
        pw.append(pk[m].mean())
    slope = np.polyfit(np.log(mids), np.log(pw), 1)[0]
    assert abs(slope + 3.0) < 0.15, slope
    # the same seed gives the same field (the workloads are reproducible)
    np.testing.assert_array_equal(f, I.gaussian_potential(n, box, seed=5, rms=1e-5))


def test_five_point_gradient_is_fourth_order():
    errs = []
    for n in (32, 64):
        box = 100.0
        x = (np.arange(n) + 0.5) * box / n
        X = np.broadcast_to(x[:, None, None], (n, n, n))
        kx = 2 * math.pi * 3 / box
        f = np.sin(kx * X)
        g = I.gradient_5pt(f, box / n)
        errs.append(np.abs(g[0] - kx * np.cos(kx * X)).max())
        assert np.abs(g[1]).max() < 1e-12 and np.abs(g[2]).max() < 1e-12
    assert 12 < errs[0] / errs[1] < 20          # halving dx divides the error by ~16


def test_refinement_fractions_full_octets_and_densest_cells():
    n, f1, ratio = 32, 0.04, 0.25
    levels, phi0, _ = I.build_field(n, 500.0, 3, f1, ratio, seed=7)
    cells0 = n ** 3
    for lev in range(1, 4):
        keys = levels[lev].keys
        assert keys.size % 8 == 0 and np.all(np.diff(keys.astype(np.int64)) > 0)
        parents = np.unique(keys >> np.uint64(3))
        assert np.array_equal(np.sort(keys), np.sort(((parents[:, None] << np.uint64(3)) +
                                                      np.arange(8, dtype=np.uint64)).ravel()))
        # parents exist on the level below
        assert np.isin(parents, levels[lev - 1].keys if lev > 1 else np.arange(cells0, dtype=np.uint64)).all()
        # volume fraction of the level: f1 * ratio^(l-1) of the box (each cell 8^-l of a coarse cell)
        frac = keys.size / 8.0 ** lev / cells0
        assert abs(frac - f1 * ratio ** (lev - 1)) < 0.2 * f1 * ratio ** (lev - 1) + 1.0 / cells0
    # level-1 parents are the densest coarse cells (delta ~ +laplacian phi)
    delta = I.spectral_laplacian(phi0, 500.0).ravel()
    ci, cj, ck = I._demorton(np.unique(levels[1].keys >> np.uint64(3)))
    chosen = delta[np.ravel_multi_index((ci, cj, ck), (n, n, n))]
    assert chosen.min() >= np.quantile(delta, 1 - f1) - 1e-12 * np.abs(delta).max()


def test_growth_normalisation_and_slices():
    assert abs(float(I.growth_over_a(1.0, 0.31)) - 1.0) < 1e-14
    g = I.growth_over_a(np.array([0.25, 0.5, 0.75]), 0.31)
    assert np.all(np.diff(g) < 0) and 1.0 < g[-1] < g[0] < 1.5   # Lambda slows growth: D+/a falls with a
    # Einstein-de Sitter: D+ ~ a, so g = 1 everywhere
    np.testing.assert_allclose(I.growth_over_a(np.array([0.3, 0.6]), 1.0), 1.0, rtol=1e-10)


def test_ray_sets():
    d = I.gnomonic_patch(16, 16, 10.0)
    np.testing.assert_allclose(np.linalg.norm(d, axis=0), 1.0, rtol=1e-14)
    ang = np.degrees(np.arccos(d[0]))            # angle from the centre (theta = 90 deg, phi = 0)
    assert ang.max() < 7.2 and ang.min() < 0.5     # corners of a 10 x 10 deg patch: ~7.07 deg
    h = I.healpix_directions(8)
    np.testing.assert_allclose(np.linalg.norm(h, axis=0), 1.0, rtol=1e-14)
    np.testing.assert_allclose(h.sum(axis=1), 0.0, atol=1e-12)   # full sky: no net direction
