"""GB300-native stage-parallel Radau IIA heat solver (arXiv 2209.06700 hot path).

Thin Python layer over the C ABI of ``libirk.so`` (include/irk.h).  PyTorch
provides device memory and streams; every step of the solver runs in libirk's
sm_103a kernels.  ``Solver`` wraps one handle.
"""
import ctypes

from . import _capi
from ._capi import (IRK_VARIANT_DIAG, IRK_VARIANT_LU, IrkError, IrkMesh, IrkOptions, IrkRequest, IrkResult,
                    IrkServeOptions, IrkStats, TABLEAU_FIELDS, ELEMENT_FIELDS, check, lib)

__all__ = ["Solver", "IrkError", "IRK_VARIANT_LU", "IRK_VARIANT_DIAG", "autotune_report", "lib", "options", "serve",
           "solve_batch", "tableau_factors", "element_factors"]


def serve(requests, max_active=8, mem_budget_bytes=0.0, realtime=True, outputs=False, max_group=0,
          reuse_handles=1, smallest_first=1, **solver_opts):
    """Run irk_serve on a list of (dim, cells, degree, Q, tau, t0, arrival_s) tuples or objects.

    Returns (status, results, ys): results are IrkResult structs, ys the host numpy arrays of
    y_{n+1} when outputs=True (else None).
    """
    import numpy as np
    n = len(requests)
    arr = (IrkRequest * n)()
    for i, r in enumerate(requests):
        if isinstance(r, tuple):
            d, N, k, Q, tau, t0, at = r
        else:
            d, N, k, Q, tau, t0, at = r.dim, r.cells, r.degree, r.Q, r.tau, 0.0, r.arrival_s
        arr[i] = IrkRequest(d, N, k, Q, float(tau), float(t0), float(at))
    o = IrkServeOptions()
    lib().irk_default_serve_options(ctypes.byref(o))
    o.max_active = int(max_active)
    o.mem_budget_bytes = float(mem_budget_bytes)
    o.realtime = 1 if realtime else 0
    o.max_group = int(max_group)
    o.reuse_handles = int(reuse_handles)
    o.smallest_first = int(smallest_first)
    for key, val in solver_opts.items():
        setattr(o.solver, key, val)
    res = (IrkResult * n)()
    ys = None
    ptrs = None
    if outputs:
        ys = []
        ptrs = (ctypes.POINTER(ctypes.c_double) * n)()
        for i in range(n):
            d, N, k = arr[i].dim, arr[i].cells, arr[i].degree
            y = np.zeros((k * N + 1) ** d)
            ys.append(y)
            ptrs[i] = y.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    status = lib().irk_serve(arr, n, ctypes.byref(o), res, ptrs)
    return status, list(res), ys


def solve_batch(solvers, ys, t_ns):
    """irk_solve_batch over Solver objects and their device vectors; returns (status, per-item statuses)."""
    n = len(solvers)
    if len(ys) != n or len(t_ns) != n:
        raise ValueError("solvers, ys and t_ns differ in length")
    hs = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    ts = (ctypes.c_double * n)(*[float(t) for t in t_ns])
    per = (ctypes.c_int * n)()
    status = lib().irk_solve_batch(hs, yp, ts, n, per)
    return status, list(per)


def tableau_factors(Q, name):
    """Factor `name` (a key of TABLEAU_FIELDS) of the Q-stage Radau IIA tableau as built on the host
    by the library (irk_tableau_factors; no device needed)."""
    import numpy as np
    size = Q if name in ("b", "c", "lam") else Q * Q
    out = (ctypes.c_double * size)()
    check(lib().irk_tableau_factors(int(Q), TABLEAU_FIELDS[name], out))
    a = np.array(out[:], dtype=np.float64)
    return a if name in ("b", "c", "lam") else a.reshape(Q, Q)


def element_factors(k, name):
    """1D element data `name` (a key of ELEMENT_FIELDS) of degree k as the library builds it on the
    host (irk_element_factors; no device needed)."""
    import numpy as np
    p = k + 1
    shape = {"nodes": (p,), "gq": (p,), "gw": (p,), "Pc": (2 * k + 1, p)}.get(name, (p, p))
    out = (ctypes.c_double * int(np.prod(shape)))()
    check(lib().irk_element_factors(int(k), ELEMENT_FIELDS[name], out))
    return np.array(out[:], dtype=np.float64).reshape(shape)


def autotune_report():
    """Launch shapes chosen so far by the operator autotuner (one line per kernel and size)."""
    n = lib().irk_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    lib().irk_autotune_report(buf, n + 1)
    return buf.value.decode()


def op_shape_force(elem_bytes, cxs=0, zc=1, cluster=0):
    """Force the launch shape of every later 3D streaming operator launch of one element size
    (4: FP32 multigrid kernels, 8: FP64-accurate kernels); cxs=0 clears the override."""
    _capi.check(lib().irk_op_shape_force(elem_bytes, cxs, zc, cluster))


def op_shape_last(elem_bytes):
    """(cxs, zc, cluster, z chunks) of the last 3D streaming operator launch of that element size."""
    out = (ctypes.c_int * 4)()
    _capi.check(lib().irk_op_shape_last(elem_bytes, out))
    return tuple(out)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def options(**kw):
    """irk_options with the library defaults, overridden by keyword arguments."""
    o = IrkOptions()
    lib().irk_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Solver:
    """One heat problem: mesh (dim, N cells per axis), degree k, Q stages, step tau."""

    def __init__(self, dim, cells, degree, Q, tau, stream=None, **opts):
        import torch
        self.dim, self.cells, self.degree, self.Q, self.tau = dim, cells, degree, Q, tau
        self.opts = options(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        mesh = IrkMesh(dim, cells)
        h = ctypes.c_void_p()
        check(lib().irk_create(ctypes.byref(mesh), degree, Q, float(tau), ctypes.byref(self.opts),
                               ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.n = lib().irk_ndofs(h)
        self.n_interior = lib().irk_ninterior(h)
        self.stride = lib().irk_stage_stride(h)
        self.levels = lib().irk_num_levels(h)

    def close(self):
        if getattr(self, "h", None):
            lib().irk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- buffers
    def vector(self, dtype=None):
        import torch
        return torch.zeros(self.n, dtype=dtype or torch.float64, device="cuda")

    def stage_vector(self, ns=None, dtype=None, level=0):
        import torch
        ns = self.Q if ns is None else ns
        stride = self.stride if level == 0 else lib().irk_level_stride(self.h, level)
        return torch.zeros(ns, stride, dtype=dtype or torch.float64, device="cuda")

    def level_ndofs(self, level):
        return lib().irk_level_ndofs(self.h, level)

    # ---- calls
    def interpolate_initial(self, y, t=0.0):
        check(lib().irk_interpolate_initial(self.h, _ptr(y), float(t)), self.h)

    def step(self, y, t_n, stage_load=None):
        st = IrkStats()
        check(lib().irk_step(self.h, _ptr(y), float(t_n), _ptr(stage_load), ctypes.byref(st)), self.h)
        return st

    def apply(self, u, v):
        check(lib().irk_apply(self.h, _ptr(u), _ptr(v)), self.h)

    def apply_op(self, u, v, Cm, Ck):
        import numpy as np
        Cm = np.ascontiguousarray(Cm, dtype=np.float64)
        Ck = np.ascontiguousarray(Ck, dtype=np.float64)
        ns = Cm.shape[0]
        check(lib().irk_apply_op(self.h, _ptr(u), _ptr(v), ns,
                                 Cm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 Ck.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.h)

    def stage_rhs(self, y, t_n, rhs):
        check(lib().irk_stage_rhs(self.h, _ptr(y), float(t_n), _ptr(rhs)), self.h)

    def precondition(self, r, z):
        check(lib().irk_precondition(self.h, _ptr(r), _ptr(z)), self.h)

    def basis_to_mg(self, r, b):
        check(lib().irk_basis_to_mg(self.h, _ptr(r), _ptr(b)), self.h)

    def basis_from_mg(self, x, z):
        check(lib().irk_basis_from_mg(self.h, _ptr(x), _ptr(z)), self.h)

    def stage_combine(self, u, v, D):
        import numpy as np
        D = np.ascontiguousarray(D, dtype=np.float64)
        check(lib().irk_stage_combine(self.h, _ptr(u), D.shape[1], _ptr(v), D.shape[0],
                                      D.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.h)

    def mg_smooth(self, level, b, x, x_is_zero):
        check(lib().irk_mg_smooth(self.h, level, _ptr(b), _ptr(x), int(x_is_zero)), self.h)

    def mg_residual(self, level, b, x, r):
        check(lib().irk_mg_residual(self.h, level, _ptr(b), _ptr(x), _ptr(r)), self.h)

    def mg_restrict(self, level, r, bc):
        check(lib().irk_mg_restrict(self.h, level, _ptr(r), _ptr(bc)), self.h)

    def mg_prolongate(self, level, ec, x):
        check(lib().irk_mg_prolongate(self.h, level, _ptr(ec), _ptr(x)), self.h)

    def mg_coarse_solve(self, b, x):
        check(lib().irk_mg_coarse_solve(self.h, _ptr(b), _ptr(x)), self.h)

    def mg_select(self, which):
        check(lib().irk_mg_select(self.h, int(which)), self.h)

    def mg_vcycle(self, level, b, x):
        check(lib().irk_mg_vcycle(self.h, level, _ptr(b), _ptr(x)), self.h)

    def tableau(self, name):
        import numpy as np
        Q = self.Q
        size = Q if name in ("b", "c", "lam") else Q * Q
        out = (ctypes.c_double * size)()
        check(lib().irk_get_tableau(self.h, TABLEAU_FIELDS[name], out), self.h)
        a = np.array(out[:], dtype=np.float64)
        return a if name in ("b", "c", "lam") else a.reshape(Q, Q)

    def cheb_interval(self, level, block):
        out = (ctypes.c_double * 2)()
        check(lib().irk_get_cheb_interval(self.h, level, block, out), self.h)
        return out[0], out[1]

    def synchronize(self):
        check(lib().irk_synchronize(self.h), self.h)


class Group(Solver):
    """R requests of one shape (dim, N cells, degree k, Q stages), each with its own step taus[r], in
    one handle: shared operator and V-cycle launches, one FGMRES per request (irk_create_group)."""

    def __init__(self, dim, cells, degree, Q, taus, stream=None, **opts):
        import torch
        self.dim, self.cells, self.degree, self.Q = dim, cells, degree, Q
        self.taus = [float(t) for t in taus]
        self.R = len(self.taus)
        self.tau = self.taus[0]
        self.opts = options(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        mesh = IrkMesh(dim, cells)
        h = ctypes.c_void_p()
        tv = (ctypes.c_double * self.R)(*self.taus)
        check(lib().irk_create_group(ctypes.byref(mesh), degree, Q, self.R, tv, ctypes.byref(self.opts),
                                     ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.n = lib().irk_ndofs(h)
        self.n_interior = lib().irk_ninterior(h)
        self.stride = lib().irk_stage_stride(h)
        self.levels = lib().irk_num_levels(h)

    def step_group(self, ys, t_ns):
        """One step of every request (ys: R device vectors, t_ns: R start times); returns
        (per-request statuses, per-request IrkStats)."""
        R = lib().irk_group_size(self.h)
        if len(ys) != R or len(t_ns) != R:
            raise ValueError("one vector and one time per request")
        ptrs = (ctypes.c_void_p * R)(*[y.data_ptr() for y in ys])
        tn = (ctypes.c_double * R)(*[float(t) for t in t_ns])
        stats = (IrkStats * R)()
        per = (ctypes.c_int * R)()
        code = lib().irk_step_group(self.h, ptrs, tn, stats, per)
        if code != _capi.IRK_OK and all(p == _capi.IRK_OK for p in per):
            check(code, self.h)
        return list(per), list(stats)

    def set_tau(self, taus):
        R = lib().irk_group_size(self.h)
        tv = (ctypes.c_double * R)(*[float(t) for t in taus])
        check(lib().irk_set_tau(self.h, tv), self.h)
        self.taus = list(tv)
        self.tau = self.taus[0]
