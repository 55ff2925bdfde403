"""Small hand-built workloads for tests (test-only helpers, no method arithmetic)."""
import dataclasses

import numpy as np

from paper_2111_08744_gb300 import inputs as I


def coarse_level_from_fn(n, box, fn, n_slices=1, slice_scale=None):
    """Level 0 with records fn(xc) -> [count, 4] at cell centres, Morton ordered."""
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    key = I.morton3(ii.ravel(), jj.ravel(), kk.ravel())
    order = np.argsort(key)
    dx = box / n
    xc = np.stack([ii.ravel(), jj.ravel(), kk.ravel()]).astype(np.float64)[:, order]
    xc = (xc + 0.5) * dx
    rec = fn(xc)
    scale = np.ones(n_slices) if slice_scale is None else np.asarray(slice_scale)
    return I.Level(keys=key[order], records=np.ascontiguousarray(rec[:, None, :] * scale[None, :, None]))


def refined_level_from_parents(parent_keys, lev, n, box, fn, n_slices=1, slice_scale=None):
    keys = ((np.asarray(parent_keys, dtype=np.uint64)[:, None] << np.uint64(3))
            | np.arange(8, dtype=np.uint64)[None, :]).ravel()
    keys = np.unique(keys)
    ci, cj, ck = I._demorton(keys)
    dx = box / (n << lev)
    xc = (np.stack([ci, cj, ck]).astype(np.float64) + 0.5) * dx
    rec = fn(xc)
    scale = np.ones(n_slices) if slice_scale is None else np.asarray(slice_scale)
    return I.Level(keys=keys, records=np.ascontiguousarray(rec[:, None, :] * scale[None, :, None]))


def random_tree(n, n_levels, box, fn, seed, frac=0.3, n_slices=1, slice_scale=None):
    """Random full-octet refinement of an n^3 grid (every refined cell has 8 children)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    levels = [coarse_level_from_fn(n, box, fn, n_slices, slice_scale)]
    for lev in range(1, n_levels + 1):
        prev = levels[-1].keys
        pick = rng.random(prev.size) < frac
        if not pick.any():
            pick[rng.integers(0, prev.size)] = True
        levels.append(refined_level_from_parents(prev[pick], lev, n, box, fn, n_slices, slice_scale))
    return levels


def workload(levels, box, n, dirs, z_max=0.5, observer=None, periodic=1, steps_per_cell=4, omega_m=0.31,
             slice_eta=None, slice_weight=None, name="custom"):
    bg = I.background_table(omega_m)
    if slice_eta is None:
        slice_eta = np.array([bg[-1, 0]])
    if slice_weight is None:
        slice_weight = np.ones(len(slice_eta))
    # default observer: near the centre but off every cell face (generic position)
    obs = (np.array([[0.5 * box + 0.137 * box / n, 0.5 * box + 0.291 * box / n, 0.5 * box + 0.443 * box / n]])
           if observer is None else np.asarray(observer, dtype=np.float64).reshape(-1, 3))
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    return I.Workload(name=name, box=box, n_coarse=n, periodic=periodic, slice_eta=np.asarray(slice_eta, float),
                      slice_weight=np.asarray(slice_weight, float), levels=levels, bg=bg, omega_m=omega_m,
                      observer=obs, z_max=np.atleast_1d(np.asarray(z_max, float)),
                      ray_begin=np.array([0, dirs.shape[1]], dtype=np.int64), dirs=dirs,
                      steps_per_cell=steps_per_cell)


def linear_fn(g, c=0.0):
    g = np.asarray(g, dtype=np.float64)

    def fn(xc):
        rec = np.empty((xc.shape[1], 4))
        rec[:, 0] = c + g @ xc
        rec[:, 1:] = g[None, :]
        return rec

    return fn


def const_fn(v):
    def fn(xc):
        rec = np.zeros((xc.shape[1], 4))
        rec[:, 0] = v
        return rec

    return fn
