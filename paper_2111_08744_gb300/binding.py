"""ctypes binding of libmt.so (include/mt.h): same names, argument marshalling only.

Every step of the ray tracing runs in the CUDA library; torch supplies device
buffers and the stream handle.  There is no CPU fallback: if libmt.so is missing
or no CUDA device is visible, `load()` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmt.so")

MT_OK, MT_ERR_INVALID_ARG, MT_ERR_OOM, MT_ERR_CUDA, MT_ERR_NOT_FULL_TREE, MT_ERR_TIMEOUT, MT_ERR_OOB, \
    MT_ERR_UNSUPPORTED = range(8)
MT_FIELD_FP64, MT_FIELD_FP32 = 0, 1
MT_INTERP_CIC, MT_INTERP_NGP, MT_INTERP_TSC = 0, 1, 2
MT_RAY_OK, MT_RAY_LEFT_DOMAIN, MT_RAY_MAX_STEPS, MT_RAY_NONFINITE = 0, 1, 2, 3
MT_HOST, MT_DEVICE_COPY, MT_DEVICE_BORROW = 0, 1, 2
MT_MAX_LEVELS, MT_MAX_SLICES, MT_MAX_CONES, MT_NOALLOC_MAX_CONES = 8, 16, 256, 4096


class MtError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} (code {code})")


class mt_grid_desc(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("n_coarse", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("n_slices", ctypes.c_int32), ("slice_eta", ctypes.c_void_p),
                ("precision", ctypes.c_int32), ("pad", ctypes.c_int32)]


class mt_level_data(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("records", ctypes.c_void_p), ("count", ctypes.c_int64),
                ("residency", ctypes.c_int32), ("pad", ctypes.c_int32)]


class mt_trace_params(ctypes.Structure):
    _fields_ = [("n_cones", ctypes.c_int32), ("steps_per_cell", ctypes.c_int32), ("gravity_on", ctypes.c_int32),
                ("interp", ctypes.c_int32), ("observer", ctypes.c_void_p), ("z_max", ctypes.c_void_p),
                ("ray_begin", ctypes.c_void_p), ("max_steps", ctypes.c_int64)]


OUT_F64 = ["x", "k", "eta", "lambda", "chi", "path", "z0", "z1", "z4", "z5", "d_a", "d_l", "phi_o", "phi_s", "isw"]
OUT_I32 = ["n_steps", "level", "status"]
OUT_ROWS = {"x": 3, "k": 4, "xi": 3}


class mt_ray_out(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in OUT_F64 + OUT_I32 + ["xi"]]


_lock = threading.Lock()
_lib = None


def load():
    """Load libmt.so (built by `paper_2111_08744_gb300.build.build()`); raise if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        lib.mt_build_octree.restype = ctypes.c_int
        lib.mt_build_octree.argtypes = [ctypes.POINTER(mt_grid_desc), ctypes.POINTER(mt_level_data), P,
                                        ctypes.c_int32, P, ctypes.POINTER(P)]
        lib.mt_trace_rays.restype = ctypes.c_int
        lib.mt_trace_rays.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64,
                                      ctypes.POINTER(mt_ray_out), P]
        lib.mt_trace_rays_adjoint.restype = ctypes.c_int
        lib.mt_trace_rays_adjoint.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64,
                                              ctypes.POINTER(mt_ray_out), P, P, P, ctypes.POINTER(P),
                                              ctypes.c_int32, P]
        lib.mt_trace_rays_jvp.restype = ctypes.c_int
        lib.mt_trace_rays_jvp.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64,
                                          ctypes.POINTER(mt_ray_out), ctypes.POINTER(P), P, P]
        lib.mt_trace_rays_lensing.restype = ctypes.c_int
        lib.mt_trace_rays_lensing.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64,
                                              ctypes.POINTER(mt_ray_out), P, P, P]
        lib.mt_trace_beams.restype = ctypes.c_int
        lib.mt_trace_beams.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_int32, ctypes.POINTER(mt_ray_out), P, P, P]
        lib.mt_find_geodesics.restype = ctypes.c_int
        lib.mt_find_geodesics.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(mt_ray_out), P, P, P, P, P, P]
        lib.mt_healpix_bin.restype = ctypes.c_int
        lib.mt_healpix_bin.argtypes = [P, ctypes.c_int64, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, P, P, P, P]
        lib.mt_deflection.restype = ctypes.c_int
        lib.mt_deflection.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64, P, P, P]
        lib.mt_field_from_coarse_phi.restype = ctypes.c_int
        lib.mt_field_from_coarse_phi.argtypes = [P, P, P, ctypes.POINTER(P), ctypes.POINTER(P), P]
        lib.mt_pullback_coarse_phi.restype = ctypes.c_int
        lib.mt_pullback_coarse_phi.argtypes = [P, ctypes.POINTER(P), P, P, P]
        lib.mt_trace_rays_noalloc.restype = ctypes.c_int
        lib.mt_trace_rays_noalloc.argtypes = [P, ctypes.POINTER(mt_trace_params), P, ctypes.c_int64,
                                              ctypes.POINTER(mt_ray_out), P]
        lib.mt_set_trace_options.restype = ctypes.c_int
        lib.mt_set_trace_options.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        lib.mt_set_launch_config.restype = ctypes.c_int
        lib.mt_set_launch_config.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        lib.mt_device_status.restype = ctypes.c_int
        lib.mt_device_status.argtypes = [P, P]
        lib.mt_free.restype = None
        lib.mt_free.argtypes = [P]
        lib.mt_status_str.restype = ctypes.c_char_p
        lib.mt_status_str.argtypes = [ctypes.c_int]
        lib.mt_octree_info.restype = ctypes.c_int
        lib.mt_octree_info.argtypes = [P, P, P]
        lib.mt_probe_fp64_fma_rate.restype = ctypes.c_int
        lib.mt_probe_fp64_fma_rate.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P]
        _lib = lib
        return lib


def status_str(code: int) -> str:
    try:
        return load().mt_status_str(int(code)).decode()
    except Exception:
        return f"status {code}"


def _check(code: int, where: str):
    if code != MT_OK:
        raise MtError(code, where)


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the ray tracer runs only on the GPU (no CPU fallback)")
    return torch


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ----------------------------------------------------------------------------- raw C-ABI names

def mt_build_octree(grid, levels, bg_table, bg_n, stream, out):
    return load().mt_build_octree(grid, levels, bg_table, bg_n, stream, out)


def mt_trace_rays(tree, params, dirs, n_rays, out, stream):
    return load().mt_trace_rays(tree, params, dirs, n_rays, out, stream)


def mt_trace_rays_adjoint(tree, params, dirs, n_rays, out, jac, lens, dL_dxi, dL_drec, checkpoint_every, stream):
    return load().mt_trace_rays_adjoint(tree, params, dirs, n_rays, out, jac, lens, dL_dxi, dL_drec,
                                        checkpoint_every, stream)


def mt_trace_rays_lensing(tree, params, dirs, n_rays, out, jac, lens, stream):
    return load().mt_trace_rays_lensing(tree, params, dirs, n_rays, out, jac, lens, stream)


def mt_trace_rays_noalloc(tree, params, dirs, n_rays, out, stream):
    return load().mt_trace_rays_noalloc(tree, params, dirs, n_rays, out, stream)


def mt_set_launch_config(tree, block_size, blocks_per_sm):
    return load().mt_set_launch_config(tree, block_size, blocks_per_sm)


def mt_device_status(tree, stream):
    return load().mt_device_status(tree, stream)


def mt_free(tree):
    load().mt_free(tree)


def mt_status_str(code):
    return status_str(code)


# ----------------------------------------------------------------------------- helpers

class Octree:
    """Owns an mt_octree handle built from a workload's levels (host numpy or CUDA tensors)."""

    def __init__(self, box, n_coarse, periodic, slice_eta, levels, bg, precision="fp32", stream=None,
                 residency=None):
        torch = _require_cuda()
        lib = load()
        self.precision = MT_FIELD_FP32 if precision in ("fp32", MT_FIELD_FP32) else MT_FIELD_FP64
        rdt = np.float32 if self.precision == MT_FIELD_FP32 else np.float64
        tdt = torch.float32 if self.precision == MT_FIELD_FP32 else torch.float64
        self._keep = []
        seta = np.ascontiguousarray(slice_eta, dtype=np.float64)
        self._keep.append(seta)
        n_levels = len(levels) - 1
        g = mt_grid_desc(float(box), int(n_coarse), n_levels, int(periodic), int(seta.size),
                         seta.ctypes.data_as(ctypes.c_void_p), self.precision, 0)
        arr = (mt_level_data * len(levels))()
        for i, lv in enumerate(levels):
            keys, rec = lv.keys, lv.records
            if isinstance(rec, torch.Tensor):
                rec = rec.to(tdt).contiguous()
                if keys is None:  # dense coarse level: keys implied
                    k = None
                else:
                    k = keys.contiguous() if isinstance(keys, torch.Tensor) else \
                        torch.from_numpy(np.ascontiguousarray(keys, dtype=np.uint64).view(np.int64)).cuda()
                self._keep += [rec] + ([k] if k is not None else [])
                arr[i] = mt_level_data(k.data_ptr() if k is not None else None, rec.data_ptr(), int(rec.shape[0]),
                                       MT_DEVICE_COPY if residency is None else residency, 0)
            else:
                k = np.ascontiguousarray(keys, dtype=np.uint64)
                r = np.ascontiguousarray(rec, dtype=rdt)
                self._keep += [k, r]
                arr[i] = mt_level_data(k.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p),
                                       int(k.size), MT_HOST, 0)
        b = np.ascontiguousarray(bg, dtype=np.float64)
        self._keep.append(b)
        h = ctypes.c_void_p()
        code = lib.mt_build_octree(ctypes.byref(g), arr, b.ctypes.data_as(ctypes.c_void_p), int(b.shape[0]),
                                   _stream_handle(stream), ctypes.byref(h))
        # host buffers may be released once the (synchronous) build returned
        self._keep = [x for x in self._keep if isinstance(x, torch.Tensor)] if residency == MT_DEVICE_BORROW else []
        _check(code, "mt_build_octree")
        self.handle = h
        self.n_levels = n_levels
        self.n_slices = int(seta.size)

    @classmethod
    def from_workload(cls, w, precision="fp32", stream=None):
        return cls(w.box, w.n_coarse, w.periodic, w.slice_eta, w.levels, w.bg, precision, stream)

    def info(self):
        cells = (ctypes.c_int64 * (self.n_levels + 1))()
        nbytes = ctypes.c_int64()
        _check(load().mt_octree_info(self.handle, cells, ctypes.byref(nbytes)), "mt_octree_info")
        return list(cells), int(nbytes.value)

    def set_trace_options(self, ray_chunk=0, staging=0):
        _check(load().mt_set_trace_options(self.handle, int(ray_chunk), int(staging)), "mt_set_trace_options")

    def set_launch_config(self, block_size=0, blocks_per_sm=0):
        _check(load().mt_set_launch_config(self.handle, int(block_size), int(blocks_per_sm)), "mt_set_launch_config")

    def device_status(self, stream=None) -> int:
        return load().mt_device_status(self.handle, _stream_handle(stream))

    def free(self):
        if getattr(self, "handle", None):
            load().mt_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


INTERP = {"cic": MT_INTERP_CIC, "ngp": MT_INTERP_NGP, "tsc": MT_INTERP_TSC}


class TraceParams:
    """Host-side cone table for mt_trace_params.  interp: "cic", "ngp" or "tsc" (or MT_INTERP_*)."""

    def __init__(self, observer, z_max, ray_begin, steps_per_cell=4, gravity_on=True, max_steps=1 << 22,
                 interp="cic"):
        self.obs = np.ascontiguousarray(np.asarray(observer, dtype=np.float64).reshape(-1, 3))
        self.zmax = np.ascontiguousarray(np.atleast_1d(np.asarray(z_max, dtype=np.float64)))
        self.begin = np.ascontiguousarray(np.asarray(ray_begin, dtype=np.int64))
        self.interp = INTERP[interp] if isinstance(interp, str) else int(interp)
        self.c = mt_trace_params(int(self.obs.shape[0]), int(steps_per_cell), 1 if gravity_on else 0, self.interp,
                                 self.obs.ctypes.data_as(ctypes.c_void_p), self.zmax.ctypes.data_as(ctypes.c_void_p),
                                 self.begin.ctypes.data_as(ctypes.c_void_p), int(max_steps))

    @classmethod
    def from_workload(cls, w, gravity_on=True, max_steps=None, steps_per_cell=None, ray_begin=None, interp="cic"):
        spc = w.steps_per_cell if steps_per_cell is None else steps_per_cell
        if max_steps is None:
            max_steps = step_cap(w.bg, w.box / w.n_coarse, len(w.levels) - 1, spc, float(np.max(w.z_max)))
        return cls(w.observer, w.z_max, w.ray_begin if ray_begin is None else ray_begin, spc, gravity_on, max_steps,
                   interp)


def step_cap(bg, dx0, n_levels, steps_per_cell, z_max):
    """A per-ray step cap from the geometry: twice the steps a ray needs if it stayed on the
    finest level all the way to z_max, plus a margin (a bound, not an estimate)."""
    a_t = 1.0 / (1.0 + z_max)
    eta = np.asarray(bg)[:, 0]
    a = np.asarray(bg)[:, 1]
    span = eta[-1] - float(np.interp(a_t, a, eta))
    return int(2.0 * span * steps_per_cell * (1 << n_levels) / dx0) + 1024


def alloc_outputs(n: int, device=None, names=None) -> Dict[str, "object"]:
    torch = _require_cuda()
    names = OUT_F64 + OUT_I32 + ["xi"] if names is None else names
    out = {}
    for k in names:
        dt = torch.int32 if k in OUT_I32 else torch.float64
        shape = (OUT_ROWS[k], n) if k in OUT_ROWS else (n,)
        out[k] = torch.empty(shape, dtype=dt, device=device or "cuda")
    return out


def ray_out_struct(out: Dict[str, "object"]) -> mt_ray_out:
    return mt_ray_out(**{k: (out[k].data_ptr() if k in out and out[k] is not None else None)
                         for k in OUT_F64 + OUT_I32 + ["xi"]})


def trace_rays(tree: Octree, params: TraceParams, dirs, out=None, stream=None):
    """mt_trace_rays on CUDA tensors: dirs float64 [3, N]; returns the output dict (device tensors)."""
    torch = _require_cuda()
    if not (isinstance(dirs, torch.Tensor) and dirs.is_cuda and dirs.dtype == torch.float64 and dirs.dim() == 2
            and dirs.shape[0] == 3 and dirs.is_contiguous()):
        raise ValueError("dirs must be a contiguous float64 CUDA tensor of shape [3, N]")
    n = int(dirs.shape[1])
    if out is None:
        out = alloc_outputs(n, dirs.device)
    o = ray_out_struct(out)
    code = load().mt_trace_rays(tree.handle, ctypes.byref(params.c), dirs.data_ptr(), n, ctypes.byref(o),
                                _stream_handle(stream))
    _check(code, "mt_trace_rays")
    return out


def trace_rays_adjoint(tree: Octree, params: TraceParams, dirs, jacobian=True, lensing=True, dL_dxi=None,
                       checkpoint_every=64, out=None, dL_drec=None, stream=None):
    """mt_trace_rays_adjoint on CUDA tensors.

    Returns the ray outputs plus "jac" [4, N] and "lens" [5, N] (forward mode) and, when dL_dxi
    ([3, N] float64 CUDA) is given, "dL_drec": one float64 tensor per level shaped like that
    level's records [count, n_slices, 4] (accumulated into `dL_drec` if passed).
    """
    torch = _require_cuda()
    n = int(dirs.shape[1])
    if out is None:
        out = alloc_outputs(n, dirs.device)
    jac = torch.empty((4, n), dtype=torch.float64, device=dirs.device) if jacobian else None
    lens = torch.empty((5, n), dtype=torch.float64, device=dirs.device) if lensing else None
    arr = None
    if dL_dxi is not None:
        if dL_drec is None:
            cells, _ = tree.info()
            dL_drec = [torch.zeros((c, tree.n_slices, 4), dtype=torch.float64, device=dirs.device) for c in cells]
        arr = (ctypes.c_void_p * len(dL_drec))(*[t.data_ptr() if t.numel() else None for t in dL_drec])
        dL_dxi = dL_dxi.contiguous()
    o = ray_out_struct(out)
    code = load().mt_trace_rays_adjoint(tree.handle, ctypes.byref(params.c), dirs.data_ptr(), n, ctypes.byref(o),
                                        jac.data_ptr() if jac is not None else None,
                                        lens.data_ptr() if lens is not None else None,
                                        dL_dxi.data_ptr() if dL_dxi is not None else None, arr,
                                        int(checkpoint_every), _stream_handle(stream))
    _check(code, "mt_trace_rays_adjoint")
    res = dict(out)
    if jac is not None:
        res["jac"] = jac
    if lens is not None:
        res["lens"] = lens
    if dL_dxi is not None:
        res["dL_drec"] = dL_drec
    return res


def mt_trace_rays_jvp(tree, params, dirs, n_rays, out, d_rec, dxi, stream):
    return load().mt_trace_rays_jvp(tree, params, dirs, n_rays, out, d_rec, dxi, stream)


def trace_rays_jvp(tree: Octree, params: TraceParams, dirs, d_rec, out=None, stream=None):
    """mt_trace_rays_jvp on CUDA tensors: the ray outputs plus "dxi" [3, N], the derivative of
    the end points on the stop surface along the record perturbation d_rec (one float64 tensor
    per level shaped like its records [count, n_slices, 4], or None for zero)."""
    torch = _require_cuda()
    n = int(dirs.shape[1])
    if out is None:
        out = alloc_outputs(n, dirs.device)
    dxi = torch.empty((3, n), dtype=torch.float64, device=dirs.device)
    keep = [t.contiguous() if t is not None else None for t in d_rec]
    arr = (ctypes.c_void_p * len(keep))(*[t.data_ptr() if (t is not None and t.numel()) else None for t in keep])
    o = ray_out_struct(out)
    code = load().mt_trace_rays_jvp(tree.handle, ctypes.byref(params.c), dirs.data_ptr(), n, ctypes.byref(o), arr,
                                    dxi.data_ptr(), _stream_handle(stream))
    _check(code, "mt_trace_rays_jvp")
    res = dict(out)
    res["dxi"] = dxi
    return res


def trace_rays_lensing(tree: Octree, params: TraceParams, dirs, out=None, stream=None):
    """mt_trace_rays_lensing on CUDA tensors: the ray outputs plus the infinitesimal-beam
    distortion matrix "jac" [4, N] and "lens" [5, N] (Eq. 12; Born approximation when the
    parameters have gravity off)."""
    torch = _require_cuda()
    n = int(dirs.shape[1])
    if out is None:
        out = alloc_outputs(n, dirs.device)
    jac = torch.empty((4, n), dtype=torch.float64, device=dirs.device)
    lens = torch.empty((5, n), dtype=torch.float64, device=dirs.device)
    o = ray_out_struct(out)
    _check(load().mt_trace_rays_lensing(tree.handle, ctypes.byref(params.c), dirs.data_ptr(), n, ctypes.byref(o),
                                        jac.data_ptr(), lens.data_ptr(), _stream_handle(stream)),
           "mt_trace_rays_lensing")
    res = dict(out)
    res["jac"] = jac
    res["lens"] = lens
    return res


def mt_trace_beams(tree, params, dirs, n_beams, eps, screen, out, jac, lens, stream):
    return load().mt_trace_beams(tree, params, dirs, n_beams, eps, screen, out, jac, lens, stream)


def trace_beams(tree: Octree, params: TraceParams, dirs, eps=1e-6, screen=0, out=None, stream=None):
    """mt_trace_beams on CUDA tensors: the central rays' outputs plus the finite-beam distortion
    matrix "jac" [4, N] and "lens" [5, N] (Eqs. 17-21; screen 0: beta-screen, 1: Sachs screen)."""
    torch = _require_cuda()
    n = int(dirs.shape[1])
    if out is None:
        out = alloc_outputs(n, dirs.device)
    jac = torch.empty((4, n), dtype=torch.float64, device=dirs.device)
    lens = torch.empty((5, n), dtype=torch.float64, device=dirs.device)
    o = ray_out_struct(out)
    _check(load().mt_trace_beams(tree.handle, ctypes.byref(params.c), dirs.data_ptr(), n, float(eps), int(screen),
                                 ctypes.byref(o), jac.data_ptr(), lens.data_ptr(), _stream_handle(stream)),
           "mt_trace_beams")
    res = dict(out)
    res["jac"] = jac
    res["lens"] = lens
    return res


def mt_find_geodesics(tree, params, src, n, tol, max_newton, max_grid, out, theta, jac, resid, iters, status, stream):
    return load().mt_find_geodesics(tree, params, src, n, tol, max_newton, max_grid, out, theta, jac, resid, iters,
                                    status, stream)


def find_geodesics(tree: Octree, params: TraceParams, src, tol=1e-9, max_newton=10, max_grid=20, stream=None):
    """mt_find_geodesics on CUDA tensors: src [3, N] source positions.  Returns the solution rays'
    outputs plus "theta" [3, N], "jac" [4, N], "resid" [N], "iters" [N] and "fstatus" [N]."""
    torch = _require_cuda()
    src = src.contiguous()
    n = int(src.shape[1])
    out = alloc_outputs(n, src.device)
    theta = torch.empty((3, n), dtype=torch.float64, device=src.device)
    jac = torch.empty((4, n), dtype=torch.float64, device=src.device)
    resid = torch.empty(n, dtype=torch.float64, device=src.device)
    iters = torch.empty(n, dtype=torch.int32, device=src.device)
    status = torch.empty(n, dtype=torch.int32, device=src.device)
    _check(load().mt_find_geodesics(tree.handle, ctypes.byref(params.c), src.data_ptr(), n, float(tol),
                                    int(max_newton), int(max_grid), ctypes.byref(ray_out_struct(out)),
                                    theta.data_ptr(), jac.data_ptr(), resid.data_ptr(), iters.data_ptr(),
                                    status.data_ptr(), _stream_handle(stream)), "mt_find_geodesics")
    res = dict(out)
    res.update(theta=theta, jac=jac, resid=resid, iters=iters, fstatus=status)
    return res


def mt_healpix_bin(dirs, n, values, k, nside, nest, sums, counts, ipix, stream):
    return load().mt_healpix_bin(dirs, n, values, k, nside, nest, sums, counts, ipix, stream)


def healpix_bin(dirs, values=None, nside=64, nest=True, stream=None):
    """mt_healpix_bin on CUDA tensors: dirs [3, N], values [K, N] (or None).  Returns
    (sums [K, 12 nside^2], counts [12 nside^2], ipix [N])."""
    torch = _require_cuda()
    dirs = dirs.contiguous()
    n = int(dirs.shape[1])
    npix = 12 * int(nside) ** 2
    k = 0 if values is None else int(values.shape[0])
    vals = None if values is None else values.contiguous().to(torch.float64)
    sums = torch.zeros((k, npix), dtype=torch.float64, device=dirs.device)
    counts = torch.zeros(npix, dtype=torch.float64, device=dirs.device)
    ipix = torch.empty(n, dtype=torch.int64, device=dirs.device)
    _check(load().mt_healpix_bin(dirs.data_ptr(), n, vals.data_ptr() if vals is not None else None, k, int(nside),
                                 1 if nest else 0, sums.data_ptr() if k else None, counts.data_ptr(), ipix.data_ptr(),
                                 _stream_handle(stream)), "mt_healpix_bin")
    return sums, counts, ipix


def deflection(tree: Octree, params: TraceParams, dirs, xi, stream=None):
    """mt_deflection: alpha [3, N] = screen components of theta - beta and the angle between them."""
    torch = _require_cuda()
    n = int(dirs.shape[1])
    alpha = torch.empty((3, n), dtype=torch.float64, device=dirs.device)
    _check(load().mt_deflection(tree.handle, ctypes.byref(params.c), dirs.contiguous().data_ptr(), n,
                                xi.contiguous().data_ptr(), alpha.data_ptr(), _stream_handle(stream)), "mt_deflection")
    return alpha


def mt_pullback_coarse_phi(tree, dL_drec, slice_weight, dL_dphi0, stream):
    return load().mt_pullback_coarse_phi(tree, dL_drec, slice_weight, dL_dphi0, stream)


def pullback_coarse_phi(tree: Octree, dL_drec, slice_weight, n_coarse, stream=None):
    """dL/dphi_0 (CUDA float64 [N_0^3], coarse Morton order) from record cotangents."""
    torch = _require_cuda()
    arr = (ctypes.c_void_p * len(dL_drec))(*[t.data_ptr() if t.numel() else None for t in dL_drec])
    w = np.ascontiguousarray(slice_weight, dtype=np.float64)
    out = torch.empty(int(n_coarse) ** 3, dtype=torch.float64, device=dL_drec[0].device)
    _check(load().mt_pullback_coarse_phi(tree.handle, arr, w.ctypes.data_as(ctypes.c_void_p), out.data_ptr(),
                                         _stream_handle(stream)), "mt_pullback_coarse_phi")
    return out


def mt_probe_fp64_fma_rate(iters, repeats, fma_per_s, stream):
    return load().mt_probe_fp64_fma_rate(iters, repeats, fma_per_s, stream)


def probe_fp64_fma_rate(iters: int = 1 << 14, repeats: int = 3, stream=None) -> float:
    """Measured FP64 FMA lane-operations per second of the current device (calibration kernel)."""
    _require_cuda()
    v = ctypes.c_double(0.0)
    _check(mt_probe_fp64_fma_rate(int(iters), int(repeats), ctypes.byref(v), _stream_handle(stream)),
           "mt_probe_fp64_fma_rate")
    return float(v.value)


def mt_field_from_coarse_phi(tree, phi0, slice_weight, base, records, stream):
    return load().mt_field_from_coarse_phi(tree, phi0, slice_weight, base, records, stream)


def field_from_coarse_phi(tree: Octree, phi0_morton, slice_weight, base=None, stream=None):
    """mt_field_from_coarse_phi on CUDA tensors: the records of every level (float64 tensors
    [count, n_slices, 4]) from the coarse potential phi0 ([N^3] float64, Morton order); base: the
    phi0-independent records per level (same shapes) or None."""
    torch = _require_cuda()
    cells, _ = tree.info()
    dev = phi0_morton.device
    recs = [torch.empty((c, tree.n_slices, 4), dtype=torch.float64, device=dev) for c in cells]
    out = (ctypes.c_void_p * len(recs))(*[t.data_ptr() if t.numel() else None for t in recs])
    bp = None
    if base is not None:
        keep = [b.contiguous() for b in base]
        bp = (ctypes.c_void_p * len(keep))(*[b.data_ptr() if b.numel() else None for b in keep])
    sw = np.ascontiguousarray(slice_weight, dtype=np.float64)
    phi = phi0_morton.contiguous()
    _check(mt_field_from_coarse_phi(tree.handle, phi.data_ptr(), sw.ctypes.data_as(ctypes.c_void_p), bp, out,
                                    _stream_handle(stream)), "mt_field_from_coarse_phi")
    return recs
