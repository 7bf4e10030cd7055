"""ctypes binding of libirk (include/irk.h): argument marshalling only.

Every computation of the solver runs in libirk's CUDA kernels; this module
loads the in-tree shared library and forwards pointers and sizes.  There is no
fallback: if libirk.so is missing or cannot be loaded, the first call into the
package raises OSError (the import itself succeeds, so that the in-package build
script can run before the library exists).
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libirk.so")

IRK_OK, IRK_EINVAL, IRK_ENOMEM, IRK_ENOTCONV, IRK_ENUMERIC, IRK_ETIMEOUT, IRK_ECUDA, IRK_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
IRK_VARIANT_LU, IRK_VARIANT_DIAG = 0, 1

ELEMENT_FIELDS = {"nodes": 0, "Me": 1, "Ke": 2, "Pc": 3, "gq": 4, "gw": 5, "B": 6, "D": 7}
TABLEAU_FIELDS = {"A": 0, "b": 1, "c": 2, "Ainv": 3, "L": 4, "U": 5, "S": 6, "Sinv": 7, "lam": 8,
                  "T": 9, "Tinv": 10, "J": 11}


class IrkMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("cells_per_axis", ctypes.c_int)]


class IrkOptions(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_it", ctypes.c_int), ("restart", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("variant", ctypes.c_int), ("mg_precision", ctypes.c_int),
                ("batched", ctypes.c_int), ("use_graph", ctypes.c_int), ("eig_steps", ctypes.c_int),
                ("smoothing_range", ctypes.c_double), ("eig_safety", ctypes.c_double),
                ("shared_cheb", ctypes.c_int), ("op_ff", ctypes.c_int), ("autotune", ctypes.c_int),
                ("pair_precond", ctypes.c_int), ("deform", ctypes.c_double),
                ("gs_reorth", ctypes.c_int)]


class IrkRequest(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("cells", ctypes.c_int), ("degree", ctypes.c_int), ("Q", ctypes.c_int),
                ("tau", ctypes.c_double), ("t0", ctypes.c_double), ("arrival_s", ctypes.c_double)]


class IrkResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("ndofs", ctypes.c_longlong), ("ninterior", ctypes.c_longlong), ("mem_bytes", ctypes.c_double),
                ("group_size", ctypes.c_int), ("handle_reused", ctypes.c_int)]


class IrkStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("vcycles", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("reorth_passes", ctypes.c_int)]


class IrkServeOptions(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("mem_budget_bytes", ctypes.c_double), ("realtime", ctypes.c_int),
                ("solver", IrkOptions), ("max_group", ctypes.c_int), ("reuse_handles", ctypes.c_int),
                ("smallest_first", ctypes.c_int)]


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong

# name -> (restype, argtypes); every symbol declared in include/irk.h
SIGNATURES = {
    "irk_default_options": (None, [ctypes.POINTER(IrkOptions)]),
    "irk_create": (_I, [ctypes.POINTER(IrkMesh), _I, _I, _D, ctypes.POINTER(IrkOptions), _P, ctypes.POINTER(_H)]),
    "irk_step": (_I, [_H, _P, _D, _P, ctypes.POINTER(IrkStats)]),
    "irk_solve_batch": (_I, [ctypes.POINTER(_H), ctypes.POINTER(_P), ctypes.POINTER(_D), _I, ctypes.POINTER(_I)]),
    "irk_destroy": (_I, [_H]),
    "irk_create_group": (_I, [ctypes.POINTER(IrkMesh), _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(IrkOptions), _P,
                             ctypes.POINTER(_H)]),
    "irk_step_group": (_I, [_H, ctypes.POINTER(_P), ctypes.POINTER(_D), ctypes.POINTER(IrkStats), ctypes.POINTER(_I)]),
    "irk_set_tau": (_I, [_H, ctypes.POINTER(_D)]),
    "irk_group_size": (_I, [_H]),
    "irk_default_serve_options": (None, [ctypes.POINTER(IrkServeOptions)]),
    "irk_serve": (_I, [ctypes.POINTER(IrkRequest), _I, ctypes.POINTER(IrkServeOptions), ctypes.POINTER(IrkResult),
                       ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]),
    "irk_ndofs": (_LL, [_H]),
    "irk_ninterior": (_LL, [_H]),
    "irk_stage_stride": (_LL, [_H]),
    "irk_num_levels": (_I, [_H]),
    "irk_strerror": (ctypes.c_char_p, [_I]),
    "irk_last_error": (ctypes.c_char_p, [_H]),
    "irk_autotune_report": (_I, [ctypes.c_char_p, _I]),
    "irk_op_shape_force": (_I, [_I, _I, _I, _I]),
    "irk_op_shape_last": (_I, [_I, ctypes.POINTER(_I)]),
    "irk_interpolate_initial": (_I, [_H, _P, _D]),
    "irk_get_tableau": (_I, [_H, _I, ctypes.POINTER(_D)]),
    "irk_tableau_factors": (_I, [_I, _I, ctypes.POINTER(_D)]),
    "irk_element_factors": (_I, [_I, _I, ctypes.POINTER(_D)]),
    "irk_get_cheb_interval": (_I, [_H, _I, _I, ctypes.POINTER(_D)]),
    "irk_apply_op": (_I, [_H, _P, _P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "irk_apply": (_I, [_H, _P, _P]),
    "irk_stage_rhs": (_I, [_H, _P, _D, _P]),
    "irk_precondition": (_I, [_H, _P, _P]),
    "irk_basis_to_mg": (_I, [_H, _P, _P]),
    "irk_basis_from_mg": (_I, [_H, _P, _P]),
    "irk_level_ndofs": (_LL, [_H, _I]),
    "irk_level_stride": (_LL, [_H, _I]),
    "irk_mg_smooth": (_I, [_H, _I, _P, _P, _I]),
    "irk_mg_residual": (_I, [_H, _I, _P, _P, _P]),
    "irk_mg_restrict": (_I, [_H, _I, _P, _P]),
    "irk_mg_restrict_noalloc": (_I, [_H, _I, _P, _P]),
    "irk_mg_prolongate": (_I, [_H, _I, _P, _P]),
    "irk_mg_coarse_solve": (_I, [_H, _P, _P]),
    "irk_mg_vcycle": (_I, [_H, _I, _P, _P]),
    "irk_mg_select": (_I, [_H, _I]),
    "irk_stage_combine": (_I, [_H, _P, _I, _P, _I, ctypes.POINTER(_D)]),
    "irk_synchronize": (_I, [_H]),
    "irk_profile": (_I, [_H, ctypes.c_uint]),
    "irk_profile_read": (_I, [_H, _I, ctypes.POINTER(_D), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
}

PROF_CATEGORIES = ["apply64", "mg_op", "mg_point", "transfer", "coarse", "combine", "krylov", "rhs", "mg_op_fine"]


class IrkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def load(path=LIB_PATH):
    """Load libirk.so and attach the signatures; raises OSError if it is missing."""
    if not os.path.exists(path):
        raise OSError(f"libirk.so not built at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(code, handle=None):
    if code != IRK_OK:
        l = lib()
        msg = l.irk_strerror(code).decode()
        if handle:
            extra = l.irk_last_error(handle)
            if extra:
                msg += ": " + extra.decode()
        raise IrkError(code, msg)
