"""FP64 CPU oracle of the null-geodesic ray tracer (arXiv 2111.08744, Sect. 2.2-2.5).

TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline / reference leg of `bench.py` may import this package.  The product
path (the CUDA library in `paper_2111_08744_gb300/` and its binding) never
imports it, and the two share no code: only the seeded input generators in
`paper_2111_08744_gb300/inputs.py` (which hold none of the method's
arithmetic) feed both.

`mt_oracle.cpp` holds the arithmetic; this module compiles it with g++
(-O2 -ffp-contract=off) and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK, STATUS_LEFT_DOMAIN, STATUS_MAX_STEPS, STATUS_NONFINITE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library (host C++17, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("n_coarse", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("n_slices", ctypes.c_int32), ("slice_eta", ctypes.c_void_p)]


class _Level(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("records", ctypes.c_void_p), ("count", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("n_cones", ctypes.c_int32), ("steps_per_cell", ctypes.c_int32), ("gravity_on", ctypes.c_int32),
                ("interp", ctypes.c_int32), ("observer", ctypes.c_void_p), ("z_max", ctypes.c_void_p),
                ("ray_begin", ctypes.c_void_p), ("max_steps", ctypes.c_int64)]


_OUT_F64 = ["x", "k", "eta", "lambda", "chi", "path", "z0", "z1", "z4", "z5", "d_a", "d_l", "phi_o", "phi_s", "isw"]
_OUT_I32 = ["n_steps", "level", "status"]


class _Out(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in _OUT_F64 + _OUT_I32 + ["tie"]]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_trace.restype = ctypes.c_int
            lib.orc_trace.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Level), ctypes.c_void_p, ctypes.c_int,
                                      ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.POINTER(_Out), ctypes.c_int]
            lib.orc_bundle.restype = ctypes.c_int
            lib.orc_bundle.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Level), ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            lib.orc_infinitesimal.restype = ctypes.c_int
            lib.orc_infinitesimal.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Level), ctypes.c_void_p,
                                              ctypes.c_int, ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p, ctypes.c_int]
            lib.orc_healpix_pixels.restype = None
            lib.orc_healpix_pixels.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                               ctypes.c_void_p]
            lib.orc_trace_to_chi.restype = ctypes.c_int
            lib.orc_trace_to_chi.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Level), ctypes.c_void_p,
                                             ctypes.c_int, ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.POINTER(_Out), ctypes.c_int]
            lib.orc_trace_analytic.restype = ctypes.c_int
            lib.orc_trace_analytic.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Level), ctypes.c_void_p,
                                               ctypes.c_int, ctypes.POINTER(_Params), ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(_Out), ctypes.c_int]
            lib.orc_sample.restype = ctypes.c_int
            lib.orc_sample.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Level), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.orc_eta_stop.restype = ctypes.c_double
            lib.orc_eta_stop.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
            lib.orc_background.restype = None
            lib.orc_background.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _Marshal:
    """Holds contiguous FP64 copies of a workload's arrays for the duration of a call."""

    def __init__(self, w, levels=None, gravity_on=True, max_steps=10_000_000, interp=0):
        lv = levels if levels is not None else w.levels
        self.keep = []
        self.seta = np.ascontiguousarray(w.slice_eta, dtype=np.float64)
        self.grid = _Grid(float(w.box), int(w.n_coarse), len(lv) - 1, int(w.periodic), int(self.seta.size),
                          _ptr(self.seta))
        arr = (_Level * len(lv))()
        for i, l in enumerate(lv):
            k = np.ascontiguousarray(l.keys, dtype=np.uint64)
            r = np.ascontiguousarray(l.records, dtype=np.float64)
            self.keep += [k, r]
            arr[i] = _Level(_ptr(k), _ptr(r), int(k.size))
        self.levels = arr
        self.bg = np.ascontiguousarray(w.bg, dtype=np.float64)
        self.obs = np.ascontiguousarray(w.observer, dtype=np.float64).reshape(-1, 3)
        self.zmax = np.ascontiguousarray(w.z_max, dtype=np.float64)
        self.begin = np.ascontiguousarray(w.ray_begin, dtype=np.int64)
        self.params = _Params(int(self.obs.shape[0]), int(w.steps_per_cell), 1 if gravity_on else 0, int(interp),
                              _ptr(self.obs), _ptr(self.zmax), _ptr(self.begin), int(max_steps))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


INTERP = {"cic": 0, "ngp": 1, "tsc": 2}


def _interp(interp):
    return INTERP[interp] if isinstance(interp, str) else int(interp)


def trace(w, dirs=None, levels=None, gravity_on=True, max_steps=10_000_000, n_threads=None, ray_begin=None,
          interp="cic", chi_stop=None, analytic=None):
    """Trace rays of workload `w` (optionally other directions / a subset). Returns a dict of arrays.

    interp: "cic" (Eq. 8), "ngp" (Eq. 7) or "tsc" (Eq. 9), each with the level fallback of Sect. 2.2.
    chi_stop: per-ray comoving distances [N]: stop on the sphere |x - x_o| = chi_stop (the geodesic
    finder's criterion, Sect. 2.5) instead of the iso-eta surface of z_max.
    analytic: (A, k_x, k_y, k_z): trace through phi = A sin(k . x) (exact, static) instead of the
    records (a smooth field for integration-order tests; the octree still sets the step size).

    Besides the per-ray outputs of the method, "tie" is the smallest margin of any index
    decision along the ray: the distance (in cell units) of a floor() argument to the
    nearest integer in a locate or CIC step, or the relative margin of the stop test.  A ray
    with a tie below ~1e-8 can take either side of a cell face under rounding alone.
    """
    lib = _load()
    m = _Marshal(w, levels, gravity_on, max_steps, _interp(interp))
    d = np.ascontiguousarray(w.dirs if dirs is None else dirs, dtype=np.float64)
    n = int(d.shape[1])
    if ray_begin is not None:
        m.begin = np.ascontiguousarray(ray_begin, dtype=np.int64)
        m.params.ray_begin = _ptr(m.begin)
    elif dirs is not None:
        if m.obs.shape[0] != 1:
            raise ValueError("pass ray_begin when tracing custom directions through several cones")
        m.begin = np.array([0, n], dtype=np.int64)
        m.params.ray_begin = _ptr(m.begin)
    out = {k: np.zeros((3, n) if k == "x" else (4, n) if k == "k" else n) for k in _OUT_F64}
    out.update({k: np.zeros(n, dtype=np.int32) for k in _OUT_I32})
    out["tie"] = np.ones(n)
    o = _Out(**{k: _ptr(v) for k, v in out.items()})
    if analytic is not None:
        an = np.ascontiguousarray(analytic, dtype=np.float64)
        rc = lib.orc_trace_analytic(ctypes.byref(m.grid), m.levels, _ptr(m.bg), int(m.bg.shape[0]),
                                    ctypes.byref(m.params), _ptr(d), n, _ptr(an), ctypes.byref(o),
                                    int(n_threads or default_threads()))
    elif chi_stop is None:
        rc = lib.orc_trace(ctypes.byref(m.grid), m.levels, _ptr(m.bg), int(m.bg.shape[0]), ctypes.byref(m.params),
                           _ptr(d), n, ctypes.byref(o), int(n_threads or default_threads()))
    else:
        cs = np.ascontiguousarray(np.broadcast_to(chi_stop, (n,)), dtype=np.float64)
        rc = lib.orc_trace_to_chi(ctypes.byref(m.grid), m.levels, _ptr(m.bg), int(m.bg.shape[0]),
                                  ctypes.byref(m.params), _ptr(d), n, _ptr(cs), ctypes.byref(o),
                                  int(n_threads or default_threads()))
    if rc != 0:
        raise RuntimeError(f"oracle trace failed with code {rc} (unsorted keys?)")
    return out


def bundle_jacobian(w, dirs=None, eps=1e-7, screen=0, levels=None, gravity_on=True, n_threads=None, interp="cic"):
    """Finite-beam distortion matrix (Eqs. 17-21) per central direction, [4, N] = A11, A12, A21, A22."""
    lib = _load()
    m = _Marshal(w, levels, gravity_on, interp=_interp(interp))
    d = np.ascontiguousarray(w.dirs if dirs is None else dirs, dtype=np.float64)
    n = int(d.shape[1])
    if dirs is not None:
        m.begin = np.array([0, n], dtype=np.int64)
        m.params.ray_begin = _ptr(m.begin)
    A = np.zeros((4, n))
    rc = lib.orc_bundle(ctypes.byref(m.grid), m.levels, _ptr(m.bg), int(m.bg.shape[0]), ctypes.byref(m.params),
                        _ptr(d), n, float(eps), int(screen), _ptr(A), int(n_threads or default_threads()))
    if rc != 0:
        raise RuntimeError(f"oracle bundle failed with code {rc}")
    return A


def infinitesimal_jacobian(w, dirs=None, levels=None, gravity_on=True, n_threads=None, interp="cic"):
    """Infinitesimal-beam distortion matrix, Eq. (12) with the Hessian of Eq. (13) and the screen
    projection of Eqs. (14)-(16) (e_1 = e_phi, e_2 = -e_theta), integrated by the trapezoidal rule
    over the step points of each traced ray.  gravity_on=False integrates along FLRW trajectories
    (the Born approximation).  Returns [4, N] = A11, A12, A21, A22."""
    lib = _load()
    m = _Marshal(w, levels, gravity_on, interp=_interp(interp))
    d = np.ascontiguousarray(w.dirs if dirs is None else dirs, dtype=np.float64)
    n = int(d.shape[1])
    if dirs is not None:
        m.begin = np.array([0, n], dtype=np.int64)
        m.params.ray_begin = _ptr(m.begin)
    A = np.zeros((4, n))
    rc = lib.orc_infinitesimal(ctypes.byref(m.grid), m.levels, _ptr(m.bg), int(m.bg.shape[0]), ctypes.byref(m.params),
                               _ptr(d), n, _ptr(A), int(n_threads or default_threads()))
    if rc != 0:
        raise RuntimeError(f"oracle infinitesimal beam failed with code {rc}")
    return A


def sample(w, pts, eta, levels=None, interp="cic"):
    """Interpolated (phi, grad[3], phi_eta, finest level, interpolation level) at points [3, n]."""
    lib = _load()
    m = _Marshal(w, levels)
    p = np.ascontiguousarray(pts, dtype=np.float64)
    n = int(p.shape[1])
    e = np.ascontiguousarray(np.broadcast_to(eta, (n,)), dtype=np.float64)
    phi, grad, pe = np.zeros(n), np.zeros((3, n)), np.zeros(n)
    lf, lc = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    rc = lib.orc_sample(ctypes.byref(m.grid), m.levels, _ptr(p), _ptr(e), n, _ptr(phi), _ptr(grad), _ptr(pe),
                        _ptr(lf), _ptr(lc), _interp(interp))
    if rc != 0:
        raise RuntimeError(f"oracle sample failed with code {rc}")
    return phi, grad, pe, lf, lc


def healpix_pixels(dirs, nside, nest=True):
    """HEALPix pixel index (NESTED or RING) of each direction [3, n] (Gorski et al. 2005)."""
    lib = _load()
    d = np.ascontiguousarray(dirs, dtype=np.float64)
    n = int(d.shape[1])
    pix = np.zeros(n, dtype=np.int64)
    lib.orc_healpix_pixels(_ptr(d), n, int(nside), 1 if nest else 0, _ptr(pix))
    return pix


def eta_stop(bg, z):
    lib = _load()
    b = np.ascontiguousarray(bg, dtype=np.float64)
    return float(lib.orc_eta_stop(_ptr(b), int(b.shape[0]), float(z)))


def background(bg, eta):
    lib = _load()
    b = np.ascontiguousarray(bg, dtype=np.float64)
    e = np.ascontiguousarray(np.atleast_1d(eta), dtype=np.float64)
    a, H = np.zeros(e.size), np.zeros(e.size)
    lib.orc_background(_ptr(b), int(b.shape[0]), _ptr(e), int(e.size), _ptr(a), _ptr(H))
    return a, H


def xi_on_surface(out, eta_stop_value):
    """End points moved along k onto the iso-eta surface eta = eta_stop ([3, N])."""
    k0 = out["k"][0]
    return out["x"] - (out["k"][1:] / k0) * (out["eta"] - eta_stop_value)
