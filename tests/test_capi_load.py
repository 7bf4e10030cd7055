"""The C-ABI library loads and exports every symbol that include/irk.h declares (CPU, no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "irk.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(irk_[a-z0-9_]+)\s*\(", text)))


def _built_lib():
    from paper_2209_06700_gb300 import _capi
    if not os.path.exists(_capi.LIB_PATH):
        from paper_2209_06700_gb300 import build
        build.build()
    return _capi


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for required in ("irk_create", "irk_step", "irk_solve_batch", "irk_destroy", "irk_apply",
                     "irk_precondition", "irk_mg_vcycle"):
        assert required in syms


def test_library_exports_every_declared_symbol():
    capi = _built_lib()
    lib = ctypes.CDLL(capi.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    capi = _built_lib()
    assert sorted(capi.SIGNATURES) == declared_symbols()
    capi.load()  # attaches every signature


def test_host_only_calls():
    capi = _built_lib()
    lib = capi.load()
    o = capi.IrkOptions()
    lib.irk_default_options(ctypes.byref(o))
    assert o.rtol == 1e-10 and o.restart == 30 and o.mg_precision == 0 and o.op_ff == 0 and o.gs_reorth == 0
    assert lib.irk_strerror(capi.IRK_ENOTCONV) == b"FGMRES did not converge"
    assert lib.irk_ndofs(None) == -1
    assert lib.irk_destroy(None) == 0
    h = ctypes.c_void_p(1234)
    out = ctypes.c_void_p()
    # invalid arguments are rejected before any device work
    assert lib.irk_create(None, 2, 2, 0.1, None, None, ctypes.byref(out)) == capi.IRK_EINVAL
    mesh = capi.IrkMesh(4, 8)
    assert lib.irk_create(ctypes.byref(mesh), 2, 2, 0.1, None, None, ctypes.byref(out)) == capi.IRK_EINVAL
    assert out.value is None
    del h


def test_op_shape_control_on_the_host():
    """irk_op_shape_force checks its ranges and irk_op_shape_last reports no launch yet (no CUDA call)."""
    capi = _built_lib()
    lib = capi.load()
    E = capi.IRK_EINVAL
    assert lib.irk_op_shape_force(2, 32, 1, 0) == E           # unknown element size
    assert lib.irk_op_shape_force(4, 12, 1, 0) == E           # segment width not 8/16/32
    assert lib.irk_op_shape_force(4, 16, 0, 0) == E           # empty z chunk
    assert lib.irk_op_shape_force(4, 16, 2, 2) == E           # cluster flag not 0/1
    out = (ctypes.c_int * 4)()
    assert lib.irk_op_shape_last(4, None) == E
    assert lib.irk_op_shape_last(3, out) == E
    assert lib.irk_op_shape_last(8, out) == capi.IRK_OK and list(out) == [-1, -1, -1, -1]
    assert lib.irk_op_shape_force(4, 16, 3, 1) == capi.IRK_OK  # valid; cleared again below
    assert lib.irk_op_shape_force(4, 0, 1, 0) == capi.IRK_OK
