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
        "irk_basis_to_mg": (N, N, N),
        "irk_basis_from_mg": (N, N, N),
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
        "irk_step_group": (N, N, d, N, N),
        "irk_set_tau": (N, d),
    }
    size_calls = {"irk_ndofs": (N,), "irk_ninterior": (N,), "irk_stage_stride": (N,), "irk_num_levels": (N,),
                  "irk_level_ndofs": (N, 0), "irk_level_stride": (N, 0), "irk_group_size": (N,)}
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


def test_create_group_refuses_bad_arguments_on_the_host(capi):
    """irk_create_group checks R, the taus and the variant before any device work."""
    lib = capi.lib()
    out = ctypes.c_void_p()
    mesh = capi.IrkMesh(3, 8)
    taus = (ctypes.c_double * 8)(*([1e-3] * 8))
    E = capi.IRK_EINVAL
    assert lib.irk_create_group(ctypes.byref(mesh), 2, 3, 2, taus, None, None, None) == E      # NULL out
    assert lib.irk_create_group(ctypes.byref(mesh), 2, 3, 2, None, None, None, ctypes.byref(out)) == E
    assert lib.irk_create_group(ctypes.byref(mesh), 2, 3, 0, taus, None, None, ctypes.byref(out)) == E
    assert out.value is None


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
    # the serving loop checks its arrays before any device query
    res = (capi.IrkResult * 1)()
    req = (capi.IrkRequest * 1)()
    assert lib.irk_serve(None, -1, None, None, None) == capi.IRK_EINVAL
    assert lib.irk_serve(None, 0, None, None, None) == capi.IRK_OK
    assert lib.irk_serve(None, 1, None, res, None) == capi.IRK_EINVAL
    assert lib.irk_serve(req, 1, None, None, None) == capi.IRK_EINVAL


def test_status_texts(capi):
    lib = capi.lib()
    codes = [capi.IRK_OK, capi.IRK_EINVAL, capi.IRK_ENOMEM, capi.IRK_ENOTCONV, capi.IRK_ENUMERIC,
             capi.IRK_ETIMEOUT, capi.IRK_ECUDA, capi.IRK_EBUSY]
    texts = [lib.irk_strerror(c) for c in codes]
    assert all(texts) and len(set(texts)) == len(codes)
    assert lib.irk_strerror(-99) == b"unknown status"


def test_create_refuses_every_documented_bad_argument(capi):
    """irk_create checks its arguments and options on the host, before any device work."""
    lib = capi.lib()
    out = ctypes.c_void_p()

    def create(dim=3, N=4, k=2, Q=3, tau=1e-2, **opt):
        o = capi.IrkOptions()
        lib.irk_default_options(ctypes.byref(o))
        for key, v in opt.items():
            setattr(o, key, v)
        mesh = capi.IrkMesh(dim, N)
        r = lib.irk_create(ctypes.byref(mesh), k, Q, tau, ctypes.byref(o), None, ctypes.byref(out))
        if r == capi.IRK_OK:   # a machine with a GPU: valid arguments create a solver
            lib.irk_destroy(out)
            out.value = None
        assert out.value is None
        return r

    E = capi.IRK_EINVAL
    assert lib.irk_create(None, 2, 2, 0.1, None, None, ctypes.byref(out)) == E
    for bad in [dict(dim=1), dict(dim=4), dict(N=0), dict(N=4097), dict(k=0), dict(k=5), dict(Q=0), dict(Q=10),
                dict(tau=0.0), dict(tau=-1e-3), dict(tau=float("inf")), dict(tau=float("nan")), dict(N=1, k=1),
                dict(rtol=0.0), dict(max_it=0), dict(restart=0), dict(restart=61), dict(cheb_degree=0),
                dict(cheb_degree=17), dict(mg_precision=16), dict(variant=2), dict(eig_steps=1),
                dict(smoothing_range=1.0), dict(eig_safety=0.9), dict(pair_precond=2), dict(deform=-0.1),
                dict(deform=0.2), dict(dim=2, deform=0.2), dict(variant=capi.IRK_VARIANT_DIAG, Q=1)]:
        assert create(**bad) == E, bad
    # control: the valid neighbours pass the host checks (without a GPU they fail later, IRK_ECUDA)
    for good in [dict(), dict(N=1, k=2), dict(dim=2, deform=0.1), dict(variant=capi.IRK_VARIANT_DIAG, Q=2),
                 dict(restart=60, cheb_degree=16, eig_steps=2, eig_safety=1.0, smoothing_range=1.5)]:
        assert create(**good) != E, good
