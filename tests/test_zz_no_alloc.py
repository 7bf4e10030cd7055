"""The allocation-free restriction entry point agrees with irk_mg_restrict.

irk_mg_restrict_noalloc serves callers that cannot allocate device memory at
this point (a serving process whose device budget is fully held by request
state, or a latency-critical loop that cannot afford a cudaMalloc/cudaFree).
It runs the same restriction with its intermediate grids in a library-owned
device array.  This file is collected last so that a run stopping at the first
failure has run every other test already; it also passes alone in a fresh
process (the first call on the device resolves the array's address).
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from paper_2209_06700_gb300 import _capi
from synthetic import uniform_vectors, zero_boundary

pytestmark = pytest.mark.gpu


def _restrict(lib, fn, s, rd, level, dt):
    bc = s.stage_vector(dtype=dt, level=level + 1)
    code = getattr(lib, fn)(s.h, level, ctypes.c_void_p(rd.data_ptr()), ctypes.c_void_p(bc.data_ptr()))
    _capi.check(code, s.h)
    s.synchronize()
    return bc.double().cpu().numpy()


@pytest.mark.parametrize("dim,N,k,Q,prec,dt", [(3, 8, 2, 3, 32, torch.float32), (2, 16, 4, 2, 32, torch.float32),
                                               (3, 12, 3, 2, 64, torch.float64)])
def test_noalloc_restrict_matches_restrict(dim, N, k, Q, prec, dt):
    lib = _capi.lib()
    with pkg.Solver(dim, N, k, Q, 1e-2, mg_precision=prec) as s:
        n1 = k * N + 1
        r = zero_boundary(uniform_vectors((Q, n1 ** dim), seed=21), dim, n1)
        rd = s.stage_vector(dtype=dt)
        rd[:, :n1 ** dim] = torch.from_numpy(r).to(dt)
        torch.cuda.synchronize()
        ref = _restrict(lib, "irk_mg_restrict", s, rd, 0, dt)
        tol = 1e-6 if prec == 32 else 1e-14
        for _ in range(2):  # two calls in a row share (and re-clear) the library's array
            got = _restrict(lib, "irk_mg_restrict_noalloc", s, rd, 0, dt)
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= tol * scale
        # a coarser level in between leaves stale data in the array; the next call still agrees
        _restrict(lib, "irk_mg_restrict_noalloc", s, s.stage_vector(dtype=dt, level=1), 1, dt)
        got = _restrict(lib, "irk_mg_restrict_noalloc", s, rd, 0, dt)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_noalloc_restrict_rejects_levels_beyond_the_array():
    lib = _capi.lib()
    # 3D degree 4 on 48^3 cells, 2 blocks: the finest restriction needs about 43 MB of intermediates
    with pkg.Solver(3, 48, 4, 2, 1e-3, restart=2) as s:
        rd = s.stage_vector(dtype=torch.float32)
        bc = s.stage_vector(dtype=torch.float32, level=1)
        code = lib.irk_mg_restrict_noalloc(s.h, 0, ctypes.c_void_p(rd.data_ptr()), ctypes.c_void_p(bc.data_ptr()))
        assert code == _capi.IRK_EINVAL
        assert b"scratch" in lib.irk_last_error(s.h)
