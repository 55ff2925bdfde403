"""Pins of the oracle's infinitesimal-beam distortion matrix (Sect. 2.3.1: Eq. 12 with the
Hessian of Eq. 13 and the screen components of Eqs. 14-16) and of its Born form (the same
integral along FLRW trajectories): a closed form for a quadratic potential, the first-order
agreement of the Born and full forms, and the correlation with the finite beams of Eq. (21)."""
import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I
from tests import helpers as H


def _quadratic_workload():
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
    return w, Q


@pytest.mark.parametrize("gravity_on", [False, True])
def test_infinitesimal_beam_quadratic_closed_form(gravity_on):
    """Constant Hessian Q: A_ab = delta_ab - 2 Q_ab int_0^chi_s (chi_s - chi) chi / chi_s dchi
    = delta_ab - (chi_s^2 / 3) e_a.Q.e_b, with e_1 = e_phi, e_2 = -e_theta of the ray direction."""
    w, Q = _quadratic_workload()
    A = oracle.infinitesimal_jacobian(w, gravity_on=gravity_on)
    chi = oracle.trace(w, gravity_on=gravity_on)["chi"]
    ref = np.empty_like(A)
    for i, r in enumerate(w.dirs.T):
        t1, t2 = np.arctan2(r[1], r[0]), np.arccos(r[2])
        e = [np.array([-np.sin(t1), np.cos(t1), 0.0]),
             np.array([-np.cos(t1) * np.cos(t2), -np.sin(t1) * np.cos(t2), np.sin(t2)])]
        for a in range(2):
            for b in range(2):
                ref[2 * a + b, i] = float(a == b) - chi[i] ** 2 / 3.0 * e[a] @ Q @ e[b]
    scale = chi.max() ** 2 / 3.0 * np.abs(Q).max()
    # trapezoidal rule on a quadratic integrand over ~150 steps: a few 1e-4 of the signal
    assert np.abs(A - ref).max() < 2e-3 * scale
    np.testing.assert_array_equal(A[1], A[2])


def test_born_and_full_agree_to_first_order_and_track_finite_beams():
    w = I.config_plain_small()
    d = np.ascontiguousarray(w.dirs[:, 5::24])
    full = oracle.infinitesimal_jacobian(w, dirs=d)
    born = oracle.infinitesimal_jacobian(w, dirs=d, gravity_on=False)
    fin = oracle.bundle_jacobian(w, dirs=d, eps=1e-6)
    k_full, k_born, k_fin = (1 - 0.5 * (a[0] + a[3]) for a in (full, born, fin))
    assert k_full.std() > 1e-3                                       # lensing is present
    # Born: the same integral on the unperturbed path, equal to first order in phi
    assert np.abs(k_born - k_full).max() < 0.2 * k_full.std()
    assert np.corrcoef(k_born, k_full)[0, 1] > 0.999
    # Eq. (12) and the finite beam of Eq. (21) measure the same convergence to leading order (the
    # finite beam on the iso-eta surface adds a radial-Hessian term): strongly correlated, slope
    # of order one, same sign
    assert np.corrcoef(k_fin, k_full)[0, 1] > 0.9
    slope = np.polyfit(k_fin, k_full, 1)[0]
    assert 0.5 < slope < 1.2, slope


def test_full_sky_mean_convergence_vanishes():
    """Over the full sky the finite-beam convergence averages to zero within its sampling error
    (a statement the paper makes about its maps; lensing conserves the total solid angle)."""
    w = I.config_plain_small()                      # full-sky HEALPix rays, nside 16
    A = oracle.bundle_jacobian(w, eps=1e-4)
    kappa = 1 - 0.5 * (A[0] + A[3])
    assert kappa.std() > 1e-3
    assert abs(kappa.mean()) < 4 * kappa.std() / np.sqrt(kappa.size)
