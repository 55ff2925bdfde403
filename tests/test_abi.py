"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/mt.h
declares, rejects invalid descriptors on the host, and the binding fails loudly without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2111_08744_gb300 import binding as B
from paper_2111_08744_gb300 import build as Bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mt_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return ctypes.CDLL(Bd.LIB)


def test_library_exports_every_declared_symbol(lib):
    syms = _declared_symbols()
    assert "mt_build_octree" in syms and "mt_trace_rays" in syms and "mt_free" in syms
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in mt.h but not exported"


def test_status_strings(lib):
    lib.mt_status_str.restype = ctypes.c_char_p
    for code in range(8):
        assert len(lib.mt_status_str(code)) > 0


def test_struct_layouts_match_header():
    # sizes implied by mt.h on LP64 (x86_64 and aarch64 alike)
    assert ctypes.sizeof(B.mt_grid_desc) == 40
    assert ctypes.sizeof(B.mt_level_data) == 32
    assert ctypes.sizeof(B.mt_trace_params) == 48
    assert ctypes.sizeof(B.mt_ray_out) == 19 * 8


def test_build_rejects_invalid_descriptors_before_gpu_work(lib):
    """Host validation returns MT_ERR_INVALID_ARG without touching the device."""
    lib.mt_build_octree.restype = ctypes.c_int
    seta = np.array([1.0])
    bg = np.zeros((4, 4))
    bg[:, 0] = np.arange(4.0)
    bg[:, 1] = 1.0
    rec = np.zeros((27, 1, 4))
    lv = (B.mt_level_data * 1)(B.mt_level_data(None, rec.ctypes.data_as(ctypes.c_void_p), 27, 0, 0))
    out = ctypes.c_void_p()
    for bad in [dict(n_coarse=3), dict(box=-1.0), dict(n_slices=0), dict(n_levels=99), dict(precision=7)]:
        d = dict(box=10.0, n_coarse=4, n_levels=0, periodic=1, n_slices=1, precision=0)
        d.update(bad)
        g = B.mt_grid_desc(d["box"], d["n_coarse"], d["n_levels"], 1, d["n_slices"],
                           seta.ctypes.data_as(ctypes.c_void_p), d["precision"], 0)
        rc = lib.mt_build_octree(ctypes.byref(g), lv, bg.ctypes.data_as(ctypes.c_void_p), 4, None,
                                 ctypes.byref(out))
        assert rc == B.MT_ERR_INVALID_ARG, bad
        assert not out.value
    # non-uniform background table
    g = B.mt_grid_desc(10.0, 4, 0, 1, 1, seta.ctypes.data_as(ctypes.c_void_p), 0, 0)
    bg2 = bg.copy()
    bg2[2, 0] = 2.5
    rc = lib.mt_build_octree(ctypes.byref(g), lv, bg2.ctypes.data_as(ctypes.c_void_p), 4, None, ctypes.byref(out))
    assert rc == B.MT_ERR_INVALID_ARG
    # incomplete octet count on a refined level
    lv2 = (B.mt_level_data * 2)(B.mt_level_data(None, rec.ctypes.data_as(ctypes.c_void_p), 64, 0, 0),
                                B.mt_level_data(None, None, 7, 0, 0))
    g = B.mt_grid_desc(10.0, 4, 1, 1, 1, seta.ctypes.data_as(ctypes.c_void_p), 0, 0)
    rc = lib.mt_build_octree(ctypes.byref(g), lv2, bg.ctypes.data_as(ctypes.c_void_p), 4, None, ctypes.byref(out))
    assert rc == B.MT_ERR_NOT_FULL_TREE


def test_trace_rejects_invalid_params(lib):
    lib.mt_trace_rays.restype = ctypes.c_int
    p = B.TraceParams([[0, 0, 0]], [1.0], [0, 10])
    o = B.mt_ray_out()
    # NULL tree
    assert lib.mt_trace_rays(None, ctypes.byref(p.c), None, 10, ctypes.byref(o), None) == B.MT_ERR_INVALID_ARG


def test_binding_fails_loudly_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        B.alloc_outputs(4)


def _declared_arity():
    """Number of parameters of every function prototype in mt.h."""
    txt = open(os.path.join(ROOT, "include", "mt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    out = {}
    for m in re.finditer(r"\b(mt_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt):
        params = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_marshals_every_entry_point_with_the_header_arity():
    """The Python binding declares, for every mt.h entry point, as many ctypes arguments as the
    prototype has parameters (the binding is argument marshalling only; a drift would pass garbage
    through the C ABI)."""
    lib = B.load()
    arity = _declared_arity()
    assert set(arity) == set(_declared_symbols())
    for name, n in arity.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, f"{name}: no argtypes in the binding"
        assert len(fn.argtypes) == n, f"{name}: binding has {len(fn.argtypes)} arguments, mt.h declares {n}"
