"""Error behaviour of the C ABI that needs no device (CPU): every call taking a handle refuses a NULL
handle with IRK_EINVAL before any CUDA call, the size queries return -1, and the batch entry point
checks its arrays (include/irk.h, conventions)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def capi():
    from tests.test_capi_load import _built_lib
    c = _built_lib()
    c.load()
    return c


def test_null_handle_is_refused_by_every_call(capi):
    lib = capi.lib()
    N = None
    d = (ctypes.c_double * 4)()
    ll = ctypes.c_longlong()
    status_calls = {
        "irk_step": (N, N, 0.0, N, N),
        "irk_interpolate_initial": (N, N, 0.0),
        "irk_get_tableau": (N, 0, d),
        "irk_get_cheb_interval": (N, 0, 0, d),
        "irk_apply_op": (N, N, N, 1, d, d),
        "irk_apply": (N, N, N),
        "irk_stage_rhs": (N, N, 0.0, N),
        "irk_precondition": (N, N, N),
        "irk_mg_smooth": (N, 0, N, N, 0),
        "irk_mg_residual": (N, 0, N, N, N),
        "irk_mg_restrict": (N, 0, N, N),
        "irk_mg_restrict_noalloc": (N, 0, N, N),
        "irk_mg_prolongate": (N, 0, N, N),
        "irk_mg_coarse_solve": (N, N, N),
        "irk_mg_vcycle": (N, 0, N, N),
        "irk_mg_select": (N, 0),
        "irk_stage_combine": (N, N, 1, N, 1, d),
        "irk_synchronize": (N,),
        "irk_profile": (N, 0),
        "irk_profile_read": (N, 0, d, ctypes.byref(ll), ctypes.byref(ll)),
    }
    size_calls = {"irk_ndofs": (N,), "irk_ninterior": (N,), "irk_stage_stride": (N,), "irk_num_levels": (N,),
                  "irk_level_ndofs": (N, 0), "irk_level_stride": (N, 0)}
    for name, args in status_calls.items():
        assert getattr(lib, name)(*args) == capi.IRK_EINVAL, name
    for name, args in size_calls.items():
        assert getattr(lib, name)(*args) == -1, name
    assert lib.irk_last_error(None) == b"NULL handle"
    assert lib.irk_destroy(None) == capi.IRK_OK
    # every entry point whose first argument is a handle is covered above
    takes_handle = {n for n, (_, args) in capi.SIGNATURES.items() if args and args[0] is ctypes.c_void_p
                    and n not in ("irk_create",)}
    assert takes_handle == set(status_calls) | set(size_calls) | {"irk_last_error", "irk_destroy"}


def test_batch_checks_its_arrays(capi):
    lib = capi.lib()
    assert lib.irk_solve_batch(None, None, None, -1, None) == capi.IRK_EINVAL
    assert lib.irk_solve_batch(None, None, None, 0, None) == capi.IRK_OK
    assert lib.irk_solve_batch(None, None, None, 1, None) == capi.IRK_EINVAL
    hs = (ctypes.c_void_p * 1)(None)
    ys = (ctypes.c_void_p * 1)(None)
    ts = (ctypes.c_double * 1)(0.0)
    per = (ctypes.c_int * 1)(12345)
    assert lib.irk_solve_batch(hs, ys, ts, 1, per) == capi.IRK_EINVAL
    assert per[0] == capi.IRK_EINVAL


def test_status_texts(capi):
    lib = capi.lib()
    codes = [capi.IRK_OK, capi.IRK_EINVAL, capi.IRK_ENOMEM, capi.IRK_ENOTCONV, capi.IRK_ENUMERIC,
             capi.IRK_ETIMEOUT, capi.IRK_ECUDA, capi.IRK_EBUSY]
    texts = [lib.irk_strerror(c) for c in codes]
    assert all(texts) and len(set(texts)) == len(codes)
    assert lib.irk_strerror(-99) == b"unknown status"
