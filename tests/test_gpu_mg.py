"""Parity of the multigrid pieces (all Q LU blocks per launch) with the oracle.

FP64 multigrid mode must agree with the oracle's plain dense implementation to
rounding (1e-12); FP32 mode to single-precision accuracy.  The Chebyshev
interval comes from the library's Lanczos estimate and is handed to the oracle,
which then runs the textbook recurrence.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.mg import (VCycle, chebyshev, jacobi_diag, level_operator, level_sizes, max_eig_DinvA,
                       prolongation)
from oracle.tableau import lu_preconditioner_factors
from synthetic import uniform_vectors, zero_boundary
from tests.gpu_util import from_dev, rel_err, to_dev

pytestmark = pytest.mark.gpu

CASES = [(2, 8, 2, 2), (2, 12, 3, 3), (3, 4, 2, 3), (3, 4, 4, 2), (3, 6, 1, 2)]
PREC = [(64, torch.float64, 1e-12), (32, torch.float32, 2e-5)]


def _blocks(Q):
    return lu_preconditioner_factors(Q)["lam"]


@pytest.mark.parametrize("dim,N,k,Q", CASES)
@pytest.mark.parametrize("prec,dt,tol", PREC)
def test_transfers_and_residual(dim, N, k, Q, prec, dt, tol):
    tau = 1e-2
    with pkg.Solver(dim, N, k, Q, tau, mg_precision=prec) as s:
        lam = _blocks(Q)
        n1f, n1c = k * N + 1, k * (N // 2) + 1
        nf, nc = n1f ** dim, n1c ** dim
        r = zero_boundary(uniform_vectors((Q, nf), seed=1), dim, n1f)
        rd = to_dev(s, r, dt)
        bc = s.stage_vector(dtype=dt, level=1)
        s.mg_restrict(0, rd, bc)
        P = prolongation(dim, N // 2, k)
        assert rel_err(from_dev(bc, nc), r @ P) <= tol
        e = zero_boundary(uniform_vectors((Q, nc), seed=2), dim, n1c)
        x0 = zero_boundary(uniform_vectors((Q, nf), seed=3), dim, n1f)
        xd = to_dev(s, x0, dt)
        s.mg_prolongate(0, to_dev(s, e, dt, level=1), xd)
        assert rel_err(from_dev(xd, nf), x0 + e @ P.T) <= tol
        b = zero_boundary(uniform_vectors((Q, nf), seed=4), dim, n1f)
        out = s.stage_vector(dtype=dt)
        s.mg_residual(0, to_dev(s, b, dt), to_dev(s, x0, dt), out)
        ref = np.stack([b[i] - level_operator(dim, N, k, lam[i], tau)[0] @ x0[i] for i in range(Q)])
        assert rel_err(from_dev(out, nf), ref) <= tol


@pytest.mark.parametrize("dim,N,k,Q", CASES)
@pytest.mark.parametrize("prec,dt,tol", PREC)
def test_smoother(dim, N, k, Q, prec, dt, tol):
    tau = 1e-2
    with pkg.Solver(dim, N, k, Q, tau, mg_precision=prec, cheb_degree=4) as s:
        lam = _blocks(Q)
        n1 = k * N + 1
        b = zero_boundary(uniform_vectors((Q, n1 ** dim), seed=7), dim, n1)
        x0 = zero_boundary(uniform_vectors((Q, n1 ** dim), seed=8), dim, n1)
        for from_zero in (True, False):
            xd = to_dev(s, np.zeros_like(x0) if from_zero else x0, dt)
            s.mg_smooth(0, to_dev(s, b, dt), xd, int(from_zero))
            got = from_dev(xd, n1 ** dim)
            ref = []
            for i in range(Q):
                A, bm = level_operator(dim, N, k, lam[i], tau)
                lo, hi = s.cheb_interval(0, i)
                start = np.zeros(n1 ** dim) if from_zero else x0[i]
                ref.append(chebyshev(A, jacobi_diag(A, bm), b[i], start, 4, lo, hi, bm))
            assert rel_err(got, np.stack(ref)) <= tol * 10


@pytest.mark.parametrize("dim,N,k,Q", CASES)
def test_chebyshev_interval_from_lanczos(dim, N, k, Q):
    """hi = 1.2 * lambda_max estimate; Lanczos never overestimates (beyond the FP32 rounding of the
    FP32 level operator it applies, about 1e-7 relative) and is within 5 %."""
    tau = 1e-2
    with pkg.Solver(dim, N, k, Q, tau) as s:
        lam = _blocks(Q)
        for i in range(Q):
            A, bm = level_operator(dim, N, k, lam[i], tau)
            true = max_eig_DinvA(A, jacobi_diag(A, bm), bm)
            lo, hi = s.cheb_interval(0, i)
            est = hi / 1.2
            assert 0.95 * true <= est <= true * (1 + 1e-6)
            assert abs(lo - hi / 10.0) <= 1e-12 * hi   # default smoothing range 10


@pytest.mark.parametrize("dim,N,k,Q", CASES)
@pytest.mark.parametrize("prec,dt,tol", PREC)
def test_vcycle(dim, N, k, Q, prec, dt, tol):
    tau = 1e-2
    with pkg.Solver(dim, N, k, Q, tau, mg_precision=prec) as s:
        lam = _blocks(Q)
        n1 = k * N + 1
        b = zero_boundary(uniform_vectors((Q, n1 ** dim), seed=9), dim, n1)
        xd = s.stage_vector(dtype=dt)
        s.mg_vcycle(0, to_dev(s, b, dt), xd)
        got = from_dev(xd, n1 ** dim)
        nlev = len(level_sizes(N, k))
        ref = []
        for i in range(Q):
            bounds = [s.cheb_interval(l, i) for l in range(nlev - 1)] + [(0.0, 1.0)]
            V = VCycle(dim, N, k, lam[i], tau, 3, bounds=bounds)
            ref.append(V.apply(b[i]))
        assert rel_err(got, np.stack(ref)) <= tol * 20


@pytest.mark.parametrize("dim,N,k,Q", CASES)
def test_coarse_solve(dim, N, k, Q):
    tau = 1e-2
    with pkg.Solver(dim, N, k, Q, tau, mg_precision=64) as s:
        lam = _blocks(Q)
        L = s.levels - 1
        Nc = level_sizes(N, k)[-1]
        n1 = k * Nc + 1
        b = zero_boundary(uniform_vectors((Q, n1 ** dim), seed=10), dim, n1)
        xd = s.stage_vector(dtype=torch.float64, level=L)
        s.mg_coarse_solve(to_dev(s, b, torch.float64, level=L), xd)
        got = from_dev(xd, n1 ** dim)
        ref = []
        for i in range(Q):
            A, bm = level_operator(dim, Nc, k, lam[i], tau)
            x = np.zeros(n1 ** dim)
            keep = ~bm
            x[keep] = np.linalg.solve(A[np.ix_(keep, keep)], b[i][keep])
            ref.append(x)
        assert rel_err(got, np.stack(ref)) <= 1e-11


@pytest.mark.parametrize("dim,N,k,Q", [(3, 5, 3, 2), (2, 37, 2, 3), (3, 9, 2, 2)])
@pytest.mark.parametrize("prec,dt", [(64, torch.float64), (32, torch.float32)])
def test_coarse_solve_fast_diagonalisation(dim, N, k, Q, prec, dt):
    """Odd coarsest meshes above 9^3 unknowns use the exact fast-diagonalisation solve."""
    tau = 1e-2
    with pkg.Solver(dim, N, k, Q, tau, mg_precision=prec) as s:
        lam = _blocks(Q)
        L = s.levels - 1
        Nc = level_sizes(N, k)[-1]
        n1 = k * Nc + 1
        assert (n1 - 2) ** dim > 729
        b = zero_boundary(uniform_vectors((Q, n1 ** dim), seed=12), dim, n1)
        xd = s.stage_vector(dtype=dt, level=L)
        s.mg_coarse_solve(to_dev(s, b, dt, level=L), xd)
        got = from_dev(xd, n1 ** dim)
        ref = []
        for i in range(Q):
            A, bm = level_operator(dim, Nc, k, lam[i], tau)
            x = np.zeros(n1 ** dim)
            keep = ~bm
            x[keep] = np.linalg.solve(A[np.ix_(keep, keep)], b[i][keep])
            ref.append(x)
        assert rel_err(got, np.stack(ref)) <= (1e-11 if prec == 64 else 2e-6)


@pytest.mark.parametrize("dim,N,k", [(2, 8, 2), (3, 4, 2), (3, 4, 3)])
@pytest.mark.parametrize("prec,dt,tol", PREC)
def test_coupled_vcycle_matches_oracle(dim, N, k, prec, dt, tol):
    """One V-cycle on the coupled 2x2 block itself (pair_precond=1, Sec. 6: GMG applied directly to
    Eq. complex:twobytwo) against the oracle's CoupledVCycle on the library's Chebyshev intervals."""
    from oracle.mg import CoupledVCycle
    from oracle.tableau import real_jordan
    Q, tau, m = 2, 1e-2, 3
    _, _, blocks = real_jordan(lu_preconditioner_factors(Q)["Ainv"])
    _, alpha, beta = blocks[0]
    n1 = k * N + 1
    n = n1 ** dim
    b = zero_boundary(uniform_vectors((2, n), seed=8), dim, n1)
    with pkg.Solver(dim, N, k, Q, tau, variant=pkg.IRK_VARIANT_DIAG, pair_precond=1, mg_precision=prec,
                    cheb_degree=m) as s:
        s.mg_select(1)
        bounds = [s.cheb_interval(lv, 0) for lv in range(len(level_sizes(N, k)) - 1)]
        xd = s.stage_vector(ns=2, dtype=dt)
        s.mg_vcycle(0, to_dev(s, b, dt), xd)
        got = from_dev(xd, n)
    ref = CoupledVCycle(dim, N, k, alpha, beta, tau, m, bounds).apply(b.reshape(-1)).reshape(2, n)
    assert rel_err(got, ref) <= tol
