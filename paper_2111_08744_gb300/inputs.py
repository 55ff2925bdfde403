"""Seeded synthetic inputs for the null-geodesic ray tracer.

This module builds the *inputs* of the method only: the background table
a(eta), H(eta) that the paper takes from the simulation's fiducial cosmology
(Sect. 2.2, "external pre-computed tables"), gridded potentials with their
gradients (Sect. 2.1, the octree "data tuple"), AMR refinement patterns,
HEALPix pixel-centre directions (Sect. 2.4, Gorski et al. 2005) and gnomonic
patches.  It contains no step of the ray tracing itself (no locate, no CIC,
no geodesic right-hand side, no integrator), so both the CUDA path and the
CPU oracle can consume what it produces without sharing method arithmetic.

Units: c = 1, lengths and conformal time in h^-1 Mpc, H0 = 1/2997.92458.

Field model (what a "refined level" holds; the synthetic stand-in for the
RAMSES light cones of Sect. 3):
  * level 0 is a dense periodic N_c^3 grid of phi_0 (Gaussian random field,
    P(k) ~ k^-3, rms fixed) and its 5-point central-difference gradient;
  * level l >= 1 cells carry
        phi_l(c)   = I_0[phi_0](x_c)   + sum_{m<l} I_m[d_m](x_c)   + d_l(c)
        grad_l(c)  = I_0[D phi_0](x_c) + sum_{m<l} I_m[D d_m](x_c) + D d_l(c)
    where I_m is trilinear interpolation of the level-m grid at the cell
    centre x_c, d_m a periodic 64^3 detail tile band-limited to level m's
    octave, and D the 5-point central stencil;
  * time slice s holds g(a_s) times the static field (g = D_+/a, g(1) = 1).
The map phi_0 -> records is linear; `coarse_records_operator_weights`
exposes the pieces the adjoint pull-back needs (slice weights).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

H0 = 1.0 / 2997.92458  # (h^-1 Mpc)^-1 with c = 1

# --------------------------------------------------------------------------
# Background cosmology (flat LCDM, no radiation)
# --------------------------------------------------------------------------

_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)


def _gl_integrate(f, lo, hi, panels=16):
    """Composite Gauss-Legendre quadrature of f over [lo, hi] (vectorised in hi)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    total = np.zeros(np.broadcast(lo, hi).shape)
    edges = [lo + (hi - lo) * (p / panels) for p in range(panels + 1)]
    for p in range(panels):
        a, b = edges[p], edges[p + 1]
        half = 0.5 * (b - a)
        mid = 0.5 * (b + a)
        for xg, wg in zip(_GL_X, _GL_W):
            total = total + wg * half * f(mid + half * xg)
    return total


def eta_of_a(a, omega_m):
    """Conformal time eta(a) = int_0^a da'/(a'^2 H(a')), flat LCDM.

    With a = s^2 the integrand becomes 2/(H0 sqrt(Om + OL s^6)), smooth on
    [0, 1], so composite Gauss-Legendre reaches machine precision.
    """
    ol = 1.0 - omega_m
    s = np.sqrt(np.asarray(a, dtype=np.float64))
    return _gl_integrate(lambda t: 2.0 / (H0 * np.sqrt(omega_m + ol * t ** 6)), 0.0, s)


def conformal_hubble(a, omega_m):
    """H_conf = a'/a = H0 sqrt(Om/a + OL a^2)."""
    ol = 1.0 - omega_m
    return H0 * np.sqrt(omega_m / a + ol * a * a)


def conformal_hubble_deta(a, omega_m):
    """d H_conf / d eta = H0^2 (2 OL a^2 - Om/a) / 2."""
    ol = 1.0 - omega_m
    return 0.5 * H0 * H0 * (2.0 * ol * a * a - omega_m / a)


def background_table(omega_m: float, z_table_max: float = 3.0, n: int = 4096) -> np.ndarray:
    """Nodes (eta_j, a_j, H_j, dH/deta_j), uniform in eta from eta(z_table_max) to eta(a=1).

    a_j is found by Newton iteration on eta(a) - eta_j with d eta/da = 1/(a H_conf).
    The last node is exactly a = 1 (today).
    """
    a_min = 1.0 / (1.0 + z_table_max)
    e_lo = float(eta_of_a(a_min, omega_m))
    e_hi = float(eta_of_a(1.0, omega_m))
    eta = e_lo + (e_hi - e_lo) * (np.arange(n, dtype=np.float64) / (n - 1))
    eta[-1] = e_hi
    # initial guess from a dense monotone sample
    a_s = np.linspace(a_min * 0.999, 1.0, 20001)
    e_s = eta_of_a(a_s, omega_m)
    a = np.interp(eta, e_s, a_s)
    for _ in range(8):
        a = a - (eta_of_a(a, omega_m) - eta) * a * conformal_hubble(a, omega_m)
    a[-1] = 1.0
    tab = np.empty((n, 4), dtype=np.float64)
    tab[:, 0] = eta
    tab[:, 1] = a
    tab[:, 2] = conformal_hubble(a, omega_m)
    tab[:, 3] = conformal_hubble_deta(a, omega_m)
    return tab


def growth_over_a(a, omega_m):
    """g(a) = D_+(a)/a normalised to g(1) = 1 (Heath 1977 integral form)."""
    ol = 1.0 - omega_m

    def dplus(av):
        av = np.asarray(av, dtype=np.float64)
        e = np.sqrt(omega_m / av ** 3 + ol)
        # int_0^a da'/(a' E)^3 with a' = t^2: integrand 2 t^4 / (Om + OL t^6)^1.5
        integ = _gl_integrate(lambda t: 2.0 * t ** 4 / (omega_m + ol * t ** 6) ** 1.5, 0.0, np.sqrt(av))
        return e * integ

    return (dplus(a) / np.asarray(a)) / (dplus(1.0) / 1.0)


# --------------------------------------------------------------------------
# HEALPix pixel centres (Gorski et al. 2005), RING and NESTED
# --------------------------------------------------------------------------

def _ring_north_index(p):
    """For p counted from the pole inside a polar cap: ring i with 2i(i-1) <= p < 2i(i+1)."""
    i = np.floor(0.5 * (1.0 + np.sqrt(1.0 + 2.0 * p))).astype(np.int64)
    i = np.where(2 * i * (i - 1) > p, i - 1, i)
    i = np.where(2 * i * (i + 1) <= p, i + 1, i)
    return i


def pix2ang_ring(nside: int, ipix) -> tuple:
    """(theta, phi) of RING pixel centres."""
    p = np.asarray(ipix, dtype=np.int64)
    n = int(nside)
    npix = 12 * n * n
    ncap = 2 * n * (n - 1)
    z = np.empty(p.shape)
    phi = np.empty(p.shape)
    north = p < ncap
    south = p >= npix - ncap
    belt = ~(north | south)
    if north.any():
        q = p[north]
        i = _ring_north_index(q)
        j = q - 2 * i * (i - 1) + 1
        z[north] = 1.0 - i * i / (3.0 * n * n)
        phi[north] = math.pi * (j - 0.5) / (2.0 * i)
    if belt.any():
        q = p[belt] - ncap
        i = q // (4 * n) + n
        j = q % (4 * n) + 1
        s = (i - n + 1) % 2
        z[belt] = 4.0 / 3.0 - 2.0 * i / (3.0 * n)
        phi[belt] = math.pi * (j - 1.0 + 0.5 * s) / (2.0 * n)
    if south.any():
        q = npix - 1 - p[south]
        i = _ring_north_index(q)
        first = npix - 2 * i * (i + 1)
        j = p[south] - first + 1
        z[south] = -(1.0 - i * i / (3.0 * n * n))
        phi[south] = math.pi * (j - 0.5) / (2.0 * i)
    return np.arccos(np.clip(z, -1.0, 1.0)), phi


def _compact_bits(v):
    """Collect the even bits of v into the low half (inverse of bit spreading by 2)."""
    v = v & 0x5555555555555555
    v = (v | (v >> 1)) & 0x3333333333333333
    v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0F
    v = (v | (v >> 4)) & 0x00FF00FF00FF00FF
    v = (v | (v >> 8)) & 0x0000FFFF0000FFFF
    v = (v | (v >> 16)) & 0x00000000FFFFFFFF
    return v


_JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4], dtype=np.int64)
_JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7], dtype=np.int64)


def pix2ang_nest(nside: int, ipix) -> tuple:
    """(theta, phi) of NESTED pixel centres via face / in-face (x, y) coordinates."""
    p = np.asarray(ipix, dtype=np.int64).astype(np.uint64)
    n = int(nside)
    npface = np.uint64(n * n)
    face = (p // npface).astype(np.int64)
    ipf = p % npface
    ix = _compact_bits(ipf).astype(np.int64)
    iy = _compact_bits(ipf >> np.uint64(1)).astype(np.int64)
    jr = _JRLL[face] * n - ix - iy - 1
    nr = np.where(jr < n, jr, np.where(jr > 3 * n, 4 * n - jr, n))
    z = np.where(jr < n, 1.0 - nr * nr / (3.0 * n * n),
                 np.where(jr > 3 * n, -(1.0 - nr * nr / (3.0 * n * n)), (2 * n - jr) * 2.0 / (3.0 * n)))
    kshift = np.where((jr >= n) & (jr <= 3 * n), (jr - n) & 1, 0)
    jp = (_JPLL[face] * nr + ix - iy + 1 + kshift) // 2
    jp = np.where(jp > 4 * n, jp - 4 * n, jp)
    jp = np.where(jp < 1, jp + 4 * n, jp)
    phi = (jp - 0.5 * (kshift + 1)) * math.pi / (2.0 * nr)
    return np.arccos(np.clip(z, -1.0, 1.0)), phi


def healpix_directions(nside: int, nest: bool = True, ipix=None) -> np.ndarray:
    """Unit vectors [3, N] of HEALPix pixel centres (all pixels unless ipix given)."""
    if ipix is None:
        ipix = np.arange(12 * nside * nside, dtype=np.int64)
    th, ph = (pix2ang_nest if nest else pix2ang_ring)(nside, ipix)
    st = np.sin(th)
    return np.stack([st * np.cos(ph), st * np.sin(ph), np.cos(th)]).astype(np.float64)


def gnomonic_patch(n1: int, n2: int, width_deg: float, theta_c: float = math.pi / 2, phi_c: float = 0.0) -> np.ndarray:
    """Unit vectors [3, n1*n2] on a tangent-plane grid n ~ c + tan(t1) e1 + tan(t2) e2.

    c is the patch centre (polar theta_c, azimuth phi_c); e1, e2 are the screen
    vectors of Sect. 2.3.2 at the centre; t1, t2 are pixel-centre offsets on a
    regular grid spanning width_deg in each direction.
    """
    c = np.array([math.cos(phi_c) * math.sin(theta_c), math.sin(phi_c) * math.sin(theta_c), math.cos(theta_c)])
    e1 = np.array([-math.sin(phi_c), math.cos(phi_c), 0.0])
    e2 = np.array([-math.cos(phi_c) * math.cos(theta_c), -math.sin(phi_c) * math.cos(theta_c), math.sin(theta_c)])
    w = math.radians(width_deg)
    t1 = (np.arange(n1) + 0.5) / n1 * w - 0.5 * w
    t2 = (np.arange(n2) + 0.5) / n2 * w - 0.5 * w
    T1, T2 = np.meshgrid(t1, t2, indexing="ij")
    v = c[:, None] + np.tan(T1).ravel()[None, :] * e1[:, None] + np.tan(T2).ravel()[None, :] * e2[:, None]
    return v / np.linalg.norm(v, axis=0, keepdims=True)


# --------------------------------------------------------------------------
# Gridded potentials
# --------------------------------------------------------------------------

def morton3(i, j, k) -> np.ndarray:
    """Morton key with x in bit 0, y in bit 1, z in bit 2 of each 3-bit group (21 bits per axis)."""

    def spread(v):
        v = np.asarray(v, dtype=np.uint64) & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v

    return spread(i) | (spread(j) << np.uint64(1)) | (spread(k) << np.uint64(2))


def _kgrid(n, box):
    kf = 2.0 * math.pi / box
    k1 = np.fft.fftfreq(n, d=1.0 / n) * kf
    kz = np.fft.rfftfreq(n, d=1.0 / n) * kf
    return k1[:, None, None], k1[None, :, None], kz[None, None, :]


def gaussian_potential(n: int, box: float, seed: int, rms: float, band: Optional[tuple] = None) -> np.ndarray:
    """Periodic Gaussian random field with P(k) ~ k^-3 (k = 0 removed), rescaled to rms exactly.

    White noise from PCG64(seed) -> FFT -> times sqrt(P(k)) -> inverse FFT.
    `band=(kmin, kmax)` keeps only kmin <= |k| < kmax (detail tiles).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    kx, ky, kz = _kgrid(n, box)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    with np.errstate(divide="ignore"):
        amp = np.where(kk > 0, kk ** -1.5, 0.0)
    if band is not None:
        amp = np.where((kk >= band[0]) & (kk < band[1]), amp, 0.0)
    f = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    f -= f.mean()
    f *= rms / math.sqrt(float(np.mean(f * f)))
    return f


def gradient_5pt(f: np.ndarray, dx: float) -> np.ndarray:
    """Periodic 5-point central gradient (f_-2 - 8 f_-1 + 8 f_+1 - f_+2) / (12 dx), shape [3, ...]."""
    out = np.empty((3,) + f.shape)
    for ax in range(3):
        out[ax] = (np.roll(f, 2, ax) - 8.0 * np.roll(f, 1, ax) + 8.0 * np.roll(f, -1, ax) - np.roll(f, -2, ax)) / (12.0 * dx)
    return out


def spectral_laplacian(f: np.ndarray, box: float) -> np.ndarray:
    n = f.shape[0]
    kx, ky, kz = _kgrid(n, box)
    return np.fft.irfftn(-(kx * kx + ky * ky + kz * kz) * np.fft.rfftn(f), s=f.shape, axes=(0, 1, 2))


def trilinear_periodic(grid: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of a periodic cell-centred grid at points u [3, M] in cell units.

    `grid` is [n, n, n] or [n, n, n, C] (channels last); returns [M] or [M, C].  Used only
    to build refined-level inputs from coarser ones (the field model above).  Runs on
    multithreaded CPU torch ops for speed; FP64 throughout.
    """
    import torch

    n = grid.shape[0]
    flat = torch.from_numpy(np.ascontiguousarray(grid).reshape(n * n * n, -1))
    v = torch.from_numpy(np.ascontiguousarray(u)) - 0.5
    i0 = torch.floor(v)
    f = v - i0
    i0 = i0.to(torch.int64)
    out = torch.zeros((u.shape[1], flat.shape[1]), dtype=torch.float64)
    for cx in (0, 1):
        wx = f[0] if cx else 1.0 - f[0]
        ix = torch.remainder(i0[0] + cx, n) * (n * n)
        for cy in (0, 1):
            wy = wx * (f[1] if cy else 1.0 - f[1])
            iy = ix + torch.remainder(i0[1] + cy, n) * n
            for cz in (0, 1):
                w = wy * (f[2] if cz else 1.0 - f[2])
                idx = iy + torch.remainder(i0[2] + cz, n)
                out += w[:, None] * flat.index_select(0, idx)
    out = out.numpy()
    return out[:, 0] if grid.ndim == 3 else out


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    keys: np.ndarray        # uint64 [count], Morton keys at this level, ascending
    records: np.ndarray     # float64 [count, n_slices, 4]: phi, dphi/dx, dphi/dy, dphi/dz


@dataclasses.dataclass
class Workload:
    name: str
    box: float
    n_coarse: int
    periodic: int
    slice_eta: np.ndarray       # ascending [S]
    slice_weight: np.ndarray    # g(a_s) per slice [S]
    levels: List[Level]
    bg: np.ndarray              # [n, 4] background table
    omega_m: float
    observer: np.ndarray        # [n_cones, 3]
    z_max: np.ndarray           # [n_cones]
    ray_begin: np.ndarray       # int64 [n_cones + 1]
    dirs: np.ndarray            # [3, N] unit vectors
    steps_per_cell: int
    phi0: Optional[np.ndarray] = None      # coarse potential (static, z = 0), [n, n, n]
    detail: Optional[list] = None          # detail tiles per refined level

    @property
    def n_levels(self):
        return len(self.levels) - 1

    @property
    def n_rays(self):
        return int(self.dirs.shape[1])

    @property
    def n_slices(self):
        return int(self.slice_eta.shape[0])


def _coarse_level(phi0, grad0, weights, n):
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    key = morton3(ii.ravel(), jj.ravel(), kk.ravel())
    order = np.argsort(key, kind="stable")
    base = np.empty((n ** 3, 4))
    base[:, 0] = phi0.ravel()
    for a in range(3):
        base[:, a + 1] = grad0[a].ravel()
    base = base[order]
    rec = base[:, None, :] * weights[None, :, None]
    return Level(keys=key[order], records=np.ascontiguousarray(rec))


def _children(keys_parent: np.ndarray) -> np.ndarray:
    """Keys of all 8 children of each parent key (octets in Morton order)."""
    return ((keys_parent[:, None] << np.uint64(3)) | np.arange(8, dtype=np.uint64)[None, :]).ravel()


def _demorton(key: np.ndarray):
    k = np.asarray(key, dtype=np.uint64)

    def compact(v):
        v = v & np.uint64(0x1249249249249249)
        v = (v | (v >> np.uint64(2))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v >> np.uint64(4))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v >> np.uint64(8))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v >> np.uint64(16))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v >> np.uint64(32))) & np.uint64(0x1FFFFF)
        return v.astype(np.int64)

    return compact(k), compact(k >> np.uint64(1)), compact(k >> np.uint64(2))


def _refined_records(keys, lev, n, box, base4, details4, tile):
    """Records (phi, grad phi) of refined level `lev` cells: trilinear interpolation of the coarse
    grid (phi_0 and its 5-point gradient, channels last in base4) at the cell centres, plus every
    coarser level's detail tile interpolated the same way, plus the level's own detail tile."""
    ci, cj, ck = _demorton(keys)
    dxl = box / (n << lev)
    xc = np.stack([ci + 0.5, cj + 0.5, ck + 0.5]).astype(np.float64) * dxl
    rec = trilinear_periodic(base4, xc / (box / n))
    for m in range(1, lev):
        rec += trilinear_periodic(details4[m - 1], xc / (box / (n << m)))
    own = details4[lev - 1]
    rec += own[ci % tile, cj % tile, ck % tile]
    return rec


def records_from_phi0(w: "Workload", phi0: np.ndarray, tile: int = 64) -> List[Level]:
    """The workload's octree (same keys) with records rebuilt from another coarse potential phi0
    (same detail tiles and slice weights): the linear field model phi0 -> records."""
    n, box = w.n_coarse, w.box
    grad0 = gradient_5pt(phi0, box / n)
    weights = np.asarray(w.slice_weight, dtype=np.float64)
    out = [_coarse_level(phi0, grad0, weights, n)]
    base4 = np.concatenate([phi0[..., None], np.moveaxis(grad0, 0, -1)], axis=-1)
    details4 = [np.concatenate([d[..., None], np.moveaxis(g, 0, -1)], axis=-1) for d, g in (w.detail or [])]
    for lev in range(1, len(w.levels)):
        keys = w.levels[lev].keys
        rec = _refined_records(keys, lev, n, box, base4, details4, tile)
        out.append(Level(keys=keys, records=np.ascontiguousarray(rec[:, None, :] * weights[None, :, None])))
    return out


def build_field(n: int, box: float, n_levels: int, f1: float, ratio: float, seed: int,
                rms: float = 1e-5, slice_weights=np.array([1.0]), tile: int = 64,
                phi0: Optional[np.ndarray] = None):
    """Coarse GRF plus `n_levels` refined levels (volume fraction f1, then f1*ratio^(l-1)).

    Returns (levels, phi0, details).  Refinement follows the density
    delta ~ +laplacian(phi) (Poisson: potential wells are over-dense), so wells refine.
    """
    dx0 = box / n
    if phi0 is None:
        phi0 = gaussian_potential(n, box, seed, rms)
    grad0 = gradient_5pt(phi0, dx0)
    weights = np.asarray(slice_weights, dtype=np.float64)
    levels = [_coarse_level(phi0, grad0, weights, n)]
    if n_levels == 0:
        return levels, phi0, []
    delta0 = spectral_laplacian(phi0, box)
    delta0 /= math.sqrt(float(np.mean(delta0 * delta0)))
    n_oct = max(1, int(round(math.log2(n / 2))))
    detail_rms = rms / math.sqrt(n_oct)
    rng_sel = np.random.Generator(np.random.PCG64(seed + 1000))
    # level-1 parents: top f1 of coarse cells by density
    flat = delta0.ravel()
    n_ref = max(1, int(round(f1 * flat.size)))
    top = np.argpartition(-flat, n_ref - 1)[:n_ref]
    ii, jj, kk = np.unravel_index(top, delta0.shape)
    parents = np.sort(morton3(ii, jj, kk))
    details = []
    details4 = []
    base4 = np.concatenate([phi0[..., None], np.moveaxis(grad0, 0, -1)], axis=-1)
    for lev in range(1, n_levels + 1):
        nl = n << lev
        dxl = box / nl
        keys = _children(parents)
        ci, cj, ck = _demorton(keys)
        # detail tile for this level: band [k_Nyq(l-1), k_Nyq(l)] of a 'tile' grid at level resolution
        tbox = tile * dxl
        knyq = math.pi / dxl
        d = gaussian_potential(tile, tbox, seed * 131 + lev, detail_rms, band=(0.5 * knyq, knyq * 1.0001))
        dgrad = gradient_5pt(d, dxl)
        details.append((d, dgrad))
        details4.append(np.concatenate([d[..., None], np.moveaxis(dgrad, 0, -1)], axis=-1))
        # cell centres in coarse units and in each detail level's units
        xc = np.stack([ci + 0.5, cj + 0.5, ck + 0.5]).astype(np.float64) * dxl  # physical
        u0 = xc / dx0
        ti, tj, tk = ci % tile, cj % tile, ck % tile
        rec = _refined_records(keys, lev, n, box, base4, details4, tile)
        levels.append(Level(keys=keys, records=np.ascontiguousarray(rec[:, None, :] * weights[None, :, None])))
        if lev == n_levels:
            break
        # choose the next parents among this level's cells
        lap = spectral_laplacian(d, tbox)
        lap /= max(1e-300, math.sqrt(float(np.mean(lap * lap))))
        dens = trilinear_periodic(delta0, u0) + 0.5 * lap[ti, tj, tk] + 1e-9 * rng_sel.standard_normal(keys.size)
        n_next = max(1, int(round(ratio * keys.size)))
        pick = np.argpartition(-dens, n_next - 1)[:n_next]
        parents = np.sort(keys[pick])
    return levels, phi0, details


def config_plain_small(n_rays_nside: int = 16) -> Workload:
    """Plain method, small: uniform 64^3 periodic grid in a 500 h^-1 Mpc box, static phi
    (GRF, P ~ k^-3, rms 1e-5), flat LCDM Om = 0.31; observer at the box centre; HEALPix
    RING nside = 16 (3072 rays) to z = 0.5; FP64 records; 10 steps per cell."""
    om = 0.31
    n, box = 64, 500.0
    levels, phi0, det = build_field(n, box, 0, 0.0, 0.0, seed=2112)
    bg = background_table(om)
    dirs = healpix_directions(n_rays_nside, nest=False)
    return Workload(
        name="plain_64cube_nside16_z0.5", box=box, n_coarse=n, periodic=1,
        slice_eta=np.array([bg[-1, 0]]), slice_weight=np.array([1.0]), levels=levels, bg=bg, omega_m=om,
        observer=np.array([[250.0, 250.0, 250.0]]), z_max=np.array([0.5]),
        ray_begin=np.array([0, dirs.shape[1]], dtype=np.int64), dirs=dirs, steps_per_cell=10,
        phi0=phi0, detail=det)


def config_amr(n: int = 256, box: float = 1000.0, n_levels: int = 3, f1: float = 0.02, ratio: float = 0.25,
               nside: int = 256, z_max: float = 1.0, seed: int = 2113, steps_per_cell: int = 4,
               ray_subset: Optional[np.ndarray] = None, name: Optional[str] = None) -> Workload:
    """AMR field: n^3 coarse grid in `box` plus `n_levels` refinement levels (factor 2 each)
    on the densest cells (f1 of the volume, then x ratio per level); refined levels carry
    added small-scale modes of the same spectrum; two time slices (z = 0 and z = 1)
    linearly interpolated in eta with phi_s = g(a_s) phi; HEALPix NESTED rays."""
    om = 0.31
    bg = background_table(om)
    a_s = np.array([0.5, 1.0])
    eta_s = eta_of_a(a_s, om)
    eta_s[-1] = bg[-1, 0]
    g = growth_over_a(a_s, om)
    levels, phi0, det = build_field(n, box, n_levels, f1, ratio, seed=seed, slice_weights=g)
    dirs = healpix_directions(nside, nest=True, ipix=ray_subset)
    return Workload(
        name=name or f"amr_{n}cube_L{n_levels}_nside{nside}_z{z_max:g}", box=box, n_coarse=n, periodic=1,
        slice_eta=eta_s, slice_weight=g, levels=levels, bg=bg, omega_m=om,
        observer=np.array([[0.5 * box, 0.5 * box, 0.5 * box]]), z_max=np.array([z_max]),
        ray_begin=np.array([0, dirs.shape[1]], dtype=np.int64), dirs=dirs, steps_per_cell=steps_per_cell,
        phi0=phi0, detail=det)


def batched_cones(base: Workload, n_cones: int = 64, n_min: float = 1e4, n_max: float = 1e6,
                  z_lo: float = 0.3, z_hi: float = 2.0, seed: int = 4113, scale: float = 1.0) -> Workload:
    """Light cones with seeded observers, z_max ~ U[z_lo, z_hi] and ray counts
    log-uniform in [n_min, n_max] (times `scale`), each a NESTED-contiguous run of
    HEALPix pixels at the smallest nside with 12 nside^2 >= count."""
    rng = np.random.Generator(np.random.PCG64(seed))
    obs = rng.uniform(0.0, base.box, size=(n_cones, 3))
    zm = rng.uniform(z_lo, z_hi, size=n_cones)
    counts = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_cones))
    counts = np.maximum(1, np.round(counts * scale)).astype(np.int64)
    dirs = []
    for c in counts:
        ns = 1
        while 12 * ns * ns < c:
            ns *= 2
        start = int(rng.integers(0, 12 * ns * ns - c + 1))
        dirs.append(healpix_directions(ns, nest=True, ipix=np.arange(start, start + c)))
    begin = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return dataclasses.replace(base, name=f"batched_{n_cones}cones", observer=obs, z_max=zm,
                               ray_begin=begin, dirs=np.concatenate(dirs, axis=1))


def with_rays(w: Workload, dirs: np.ndarray, name: Optional[str] = None) -> Workload:
    """Same field and single cone, different ray directions."""
    return dataclasses.replace(w, dirs=np.ascontiguousarray(dirs),
                               ray_begin=np.array([0, dirs.shape[1]], dtype=np.int64), name=name or w.name)


def cached(builder, cache_dir: Optional[str] = None, **kwargs) -> Workload:
    """builder(**kwargs), memoised on disk (pickle) under cache_dir or $MT_WORKLOAD_CACHE.

    Generation of the large AMR fields takes tens of seconds; repeated processes on one
    machine (tests, benchmark, profiler runs) reuse the pickled result.  No cache is used
    when neither is set.
    """
    import hashlib
    import os
    import pickle

    d = cache_dir or os.environ.get("MT_WORKLOAD_CACHE")
    if not d:
        return builder(**kwargs)
    key = hashlib.sha1(repr((builder.__name__, sorted(kwargs.items()))).encode()).hexdigest()[:16]
    path = os.path.join(d, f"{builder.__name__}_{key}.pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    w = builder(**kwargs)
    os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        pickle.dump(w, f, protocol=pickle.HIGHEST_PROTOCOL)
    os.replace(tmp, path)
    return w


def fp32_levels(w: Workload) -> List[Level]:
    """The same records rounded to float32 (the mixed-precision field)."""
    return [Level(keys=l.keys, records=l.records.astype(np.float32)) for l in w.levels]


# --------------------------------------------------------------------------
# Large workloads generated on the GPU (same field model, torch CUDA tensors)
# --------------------------------------------------------------------------

def _t_morton(i, j, k):
    """Morton keys of int64 CUDA tensors (same bit layout as morton3)."""
    import torch

    def spread(v):
        v = v & 0x1FFFFF
        v = (v | (v << 32)) & 0x1F00000000FFFF
        v = (v | (v << 16)) & 0x1F0000FF0000FF
        v = (v | (v << 8)) & 0x100F00F00F00F00F
        v = (v | (v << 4)) & 0x10C30C30C30C30C3
        v = (v | (v << 2)) & 0x1249249249249249
        return v

    return spread(i) | (spread(j) << 1) | (spread(k) << 2)


def _t_demorton(key):
    def compact(v):
        v = v & 0x1249249249249249
        v = (v | (v >> 2)) & 0x10C30C30C30C30C3
        v = (v | (v >> 4)) & 0x100F00F00F00F00F
        v = (v | (v >> 8)) & 0x1F0000FF0000FF
        v = (v | (v >> 16)) & 0x1F00000000FFFF
        v = (v | (v >> 32)) & 0x1FFFFF
        return v

    return compact(key), compact(key >> 1), compact(key >> 2)


def _t_trilinear(grid, xc_units):
    """Trilinear interpolation of a periodic cell-centred [n, n, n] CUDA grid at points [3, M]
    given in cell units (FP32 weights); chunked to bound temporaries."""
    import torch
    n = grid.shape[0]
    flat = grid.reshape(-1)
    out = torch.empty(xc_units.shape[1], dtype=grid.dtype, device=grid.device)
    step = 1 << 25
    for a in range(0, xc_units.shape[1], step):
        u = xc_units[:, a:a + step] - 0.5
        i0 = torch.floor(u)
        f = (u - i0).to(grid.dtype)
        i0 = i0.to(torch.int64)
        acc = torch.zeros(u.shape[1], dtype=grid.dtype, device=grid.device)
        for cx in (0, 1):
            wx = f[0] if cx else 1 - f[0]
            ix = ((i0[0] + cx) % n) * (n * n)
            for cy in (0, 1):
                wy = wx * (f[1] if cy else 1 - f[1])
                iy = ix + ((i0[1] + cy) % n) * n
                for cz in (0, 1):
                    w = wy * (f[2] if cz else 1 - f[2])
                    acc += w * flat[iy + ((i0[2] + cz) % n)]
        out[a:a + step] = acc
    return out


def _t_threshold(values, frac, seed, sample=1 << 23):
    """Value above which about `frac` of `values` lie (quantile of a seeded subsample)."""
    import torch
    g = torch.Generator(device=values.device)
    g.manual_seed(seed)
    idx = torch.randint(0, values.numel(), (min(sample, values.numel()),), generator=g, device=values.device)
    return torch.quantile(values.reshape(-1)[idx].float(), 1.0 - frac).item()


@dataclasses.dataclass
class GpuLevel:
    keys: "object"      # int64 CUDA tensor (Morton keys), None for the dense coarse level
    records: "object"   # float32 CUDA tensor [count, n_slices, 4]


def config_large_gpu(n: int = 1024, box: float = 2600.0, n_levels: int = 4, f1: float = 0.03, ratio: float = 0.125,
                     nside: int = 2048, z_max: float = 2.0, seed: int = 2115, steps_per_cell: int = 4,
                     slice_z=(2.0, 1.0, 0.5, 0.0), rms: float = 1e-5, tile: int = 64, device: str = "cuda",
                     ray_subset: Optional[np.ndarray] = None):
    """The large AMR workload built on the GPU: n^3 coarse grid plus n_levels refined levels
    (volume fraction f1, then x ratio per level), len(slice_z) time slices, HEALPix NESTED rays.
    Same field model as build_field (records in FP32): coarse GRF phi_0 from PCG64 white noise,
    5-point gradient, refined records = trilinear interpolation of the coarse grid at the cell
    centre + coarser detail tiles + the level's own detail tile, slice s scaled by g(a_s)."""
    import torch
    dev = torch.device(device)
    om = 0.31
    bg = background_table(om)
    a_s = 1.0 / (1.0 + np.asarray(slice_z, dtype=np.float64))
    order = np.argsort(a_s)
    a_s = a_s[order]
    eta_s = eta_of_a(a_s, om)
    if a_s[-1] == 1.0:
        eta_s[-1] = bg[-1, 0]
    gw = growth_over_a(a_s, om)
    wt = torch.tensor(gw, dtype=torch.float32, device=dev)
    dx0 = box / n
    # coarse GRF: PCG64 white noise -> FFT -> sqrt(P(k)), P ~ k^-3 -> rms
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    for i in range(n):
        phi[i] = torch.from_numpy(rng.standard_normal((n, n), dtype=np.float32)).to(dev)
    kf = 2.0 * math.pi / box
    k1 = torch.fft.fftfreq(n, d=1.0 / n, device=dev) * kf
    kz = torch.fft.rfftfreq(n, d=1.0 / n, device=dev) * kf
    fk = torch.fft.rfftn(phi)
    del phi
    for i in range(n):  # in place, plane by plane: amplitude k^-1.5, k = 0 removed
        kk = torch.sqrt(k1[i] ** 2 + k1[:, None] ** 2 + kz[None, :] ** 2)
        amp = torch.where(kk > 0, kk.clamp_min(1e-30) ** -1.5, torch.zeros_like(kk))
        fk[i] *= amp
    phi0 = torch.fft.irfftn(fk, s=(n, n, n))
    # density estimate for refinement: +laplacian (spectral), unit variance
    for i in range(n):
        fk[i] *= -(k1[i] ** 2 + k1[:, None] ** 2 + kz[None, :] ** 2)
    delta = torch.fft.irfftn(fk, s=(n, n, n))
    del fk
    phi0 -= phi0.mean()
    phi0 *= rms / torch.sqrt((phi0.double() ** 2).mean()).float()
    delta /= torch.sqrt((delta.double() ** 2).mean()).float()
    grad0 = [(torch.roll(phi0, 2, ax) - 8.0 * torch.roll(phi0, 1, ax) + 8.0 * torch.roll(phi0, -1, ax)
              - torch.roll(phi0, -2, ax)) / (12.0 * dx0) for ax in range(3)]
    # level 0: records in Morton order, [count, S, 4]
    S = len(a_s)
    n0 = n ** 3
    rec0 = torch.empty((n0, S, 4), dtype=torch.float32, device=dev)
    ar = torch.arange(n, device=dev, dtype=torch.int64)
    for i in range(n):
        jj, kk = torch.meshgrid(ar, ar, indexing="ij")
        keys = _t_morton(torch.full_like(jj, i), jj, kk).reshape(-1)
        vals = torch.empty((n * n, 4), dtype=torch.float32, device=dev)
        vals[:, 0] = phi0[i].reshape(-1)
        for ax in range(3):
            vals[:, 1 + ax] = grad0[ax][i].reshape(-1)
        rec0[keys] = vals[:, None, :] * wt[None, :, None]
    levels = [GpuLevel(keys=None, records=rec0)]
    # refined levels
    thr = _t_threshold(delta, f1, seed)
    sel = torch.nonzero(delta.reshape(-1) > thr).squeeze(1)
    ci, cj, ck = sel // (n * n), (sel // n) % n, sel % n
    parents = torch.sort(_t_morton(ci, cj, ck)).values
    del sel, ci, cj, ck
    n_oct = max(1, int(round(math.log2(n / 2))))
    detail_rms = rms / math.sqrt(n_oct)
    details = []
    for lev in range(1, n_levels + 1):
        dxl = box / (n << lev)
        keys = ((parents[:, None] << 3) | torch.arange(8, device=dev)[None, :]).reshape(-1)
        d = gaussian_potential(tile, tile * dxl, seed * 131 + lev, detail_rms,
                               band=(0.5 * math.pi / dxl, math.pi / dxl * 1.0001))
        dgrad = gradient_5pt(d, dxl)
        dt = torch.from_numpy(d.astype(np.float32)).to(dev)
        dgt = torch.from_numpy(dgrad.astype(np.float32)).to(dev)
        details.append((dt, dgt))
        cnt = keys.numel()
        rec = torch.empty((cnt, S, 4), dtype=torch.float32, device=dev)
        step = 1 << 26
        dens_all = torch.empty(cnt, dtype=torch.float32, device=dev) if lev < n_levels else None
        if dens_all is not None:
            lap = torch.from_numpy(spectral_laplacian(d, tile * dxl).astype(np.float32)).to(dev)
            lap /= torch.sqrt((lap.double() ** 2).mean()).float()
        for a in range(0, cnt, step):
            kc = keys[a:a + step]
            ci, cj, ck = _t_demorton(kc)
            xc = (torch.stack([ci, cj, ck]).double() + 0.5) * dxl
            vals = torch.empty((kc.numel(), 4), dtype=torch.float32, device=dev)
            u0 = xc / dx0
            vals[:, 0] = _t_trilinear(phi0, u0)
            for ax in range(3):
                vals[:, 1 + ax] = _t_trilinear(grad0[ax], u0)
            for m in range(1, lev):
                dm, dgm = details[m - 1]
                um = xc / (box / (n << m))
                vals[:, 0] += _t_trilinear(dm, um)
                for ax in range(3):
                    vals[:, 1 + ax] += _t_trilinear(dgm[ax], um)
            ti, tj, tk = ci % tile, cj % tile, ck % tile
            vals[:, 0] += dt[ti, tj, tk]
            for ax in range(3):
                vals[:, 1 + ax] += dgt[ax][ti, tj, tk]
            rec[a:a + step] = vals[:, None, :] * wt[None, :, None]
            if dens_all is not None:
                dens_all[a:a + step] = _t_trilinear(delta, u0) + 0.5 * lap[ti, tj, tk]
        levels.append(GpuLevel(keys=keys, records=rec))
        if lev == n_levels:
            break
        thr = _t_threshold(dens_all, ratio, seed + lev)
        parents = torch.sort(keys[dens_all > thr]).values
        del dens_all
    del delta, grad0
    dirs = healpix_directions(nside, nest=True, ipix=ray_subset)
    w = Workload(name=f"large_{n}cube_L{n_levels}_nside{nside}_z{z_max:g}", box=box, n_coarse=n, periodic=1,
                 slice_eta=eta_s, slice_weight=gw, levels=levels, bg=bg, omega_m=om,
                 observer=np.array([[0.5 * box] * 3]), z_max=np.array([z_max]),
                 ray_begin=np.array([0, dirs.shape[1]], dtype=np.int64), dirs=dirs, steps_per_cell=steps_per_cell,
                 phi0=None, detail=None)
    return w


def config_diff(n_pix: int = 1024, n: int = 128, box: float = 1000.0, n_levels: int = 3, width_deg: float = 10.0,
                z_max: float = 1.0, seed: int = 2114) -> Workload:
    """Differentiation workload: the AMR generator at n^3 coarse cells in `box` (3 levels, two
    slices), n_pix x n_pix rays on a tangent-plane grid of width_deg centred on (theta = 90 deg,
    phi = 0) to z_max; the end-point loss is compared with the FLRW end points."""
    w = config_amr(n=n, box=box, n_levels=n_levels, nside=1, z_max=z_max, seed=seed, name="diff")
    dirs = gnomonic_patch(n_pix, n_pix, width_deg)
    return with_rays(w, dirs, name=f"diff_{n}cube_L{n_levels}_{n_pix}x{n_pix}_z{z_max:g}")
