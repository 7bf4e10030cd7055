"""Oracle pins for the IRK step (CPU only).

Pins: Q=1 reduces to backward Euler written out by hand; three independent
exact routes agree (sparse direct Kronecker solve, per-mode fast
diagonalisation, transformed system Eq. (irk:A) solved directly); the
temporal order 2Q-1 (Sec. 2) against the closed-form semi-discrete
solution; the spatial order k+1 against the manufactured solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.fem import assemble, interior_restrict
from oracle.heat import l2_error, phi_time
from oracle.irk import (FastDiag, Problem, apply_calA, exact_semidiscrete, run_steps, step_direct,
                        step_fastdiag)


def test_q1_is_backward_euler():
    prob = Problem(2, 4, 2, 1, 0.05)
    mesh = prob.mesh
    M, K = assemble(mesh)
    MI, keep = interior_restrict(mesh, M)
    KI, _ = interior_restrict(mesh, K)
    y0 = prob.y0()
    t = 0.3
    # (M + tau K) y1 = M y0 + tau g(t + tau)
    rhs = MI @ y0[keep] + prob.tau * phi_time(2, t + prob.tau) * prob.G[keep]
    y1 = spla.spsolve((MI + prob.tau * KI).tocsc(), rhs)
    got = step_direct(prob, y0, t)
    np.testing.assert_allclose(got[keep], y1, rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,N,k,Q,tau", [(2, 4, 2, 2, 0.05), (2, 3, 3, 3, 0.01), (3, 2, 2, 3, 0.01),
                                         (3, 3, 1, 4, 0.1), (2, 2, 4, 5, 0.002)])
def test_direct_equals_fastdiag(d, N, k, Q, tau):
    prob = Problem(d, N, k, Q, tau)
    rng = np.random.default_rng(1)
    y = prob.y0() + 0.1 * rng.uniform(-1, 1, prob.mesh.n)
    y[prob.mesh.boundary_mask()] = 0.0
    a = step_direct(prob, y, 0.2)
    b = step_fastdiag(prob, y, 0.2)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_transformed_system_same_solution():
    """Eq. (irk:A): calA k = (A^{-1} (x) I)(gbar - 1 (x) K y_n) has the same k."""
    prob = Problem(2, 3, 2, 3, 0.02)
    mesh = prob.mesh
    y0 = prob.y0()
    _, k_ref = step_direct(prob, y0, 0.1, return_stages=True)
    keep = np.flatnonzero(~mesh.boundary_mask())
    # assemble calA column by column through apply_calA (the matrix-free definition)
    n = mesh.n
    Q = prob.Q
    cols = []
    for q in range(Q):
        for j in keep:
            e = np.zeros((Q, n))
            e[q, j] = 1.0
            cols.append(apply_calA(prob, e)[:, keep].reshape(-1))
    calA = np.array(cols).T
    rhs = prob.stage_rhs_calA(y0, 0.1)[:, keep].reshape(-1)
    k = np.linalg.solve(calA, rhs).reshape(Q, -1)
    assert np.abs(k - k_ref[:, keep]).max() <= 1e-11 * np.abs(k_ref).max()
    # and calA (x) equals the Kronecker assembly A^{-1} (x) M + tau I (x) K
    M, K = assemble(mesh)
    MI, _ = interior_restrict(mesh, M)
    KI, _ = interior_restrict(mesh, K)
    kron = (sp.kron(sp.csr_matrix(prob.Ainv), MI) + prob.tau * sp.kron(sp.identity(Q), KI)).toarray()
    assert np.abs(kron - calA).max() <= 1e-14 * np.abs(kron).max() * 10


@pytest.mark.parametrize("Q", [1, 2, 3])
def test_temporal_order(Q):
    errs = []
    steps = [8, 16, 32]
    for nst in steps:
        prob = Problem(2, 4, 2, Q, 1.0 / nst)
        fd = FastDiag(prob)
        y = run_steps(prob, nst)
        ex = exact_semidiscrete(prob, prob.y0(), 1.0, fd)
        errs.append(np.abs(y - ex).max())
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - (2 * Q - 1)) < 0.2, (errs, rate)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_spatial_order(k):
    errs = []
    for N in [4, 8, 16]:
        prob = Problem(2, N, k, 5, 0.05)
        y = run_steps(prob, 4)
        errs.append(l2_error(prob.mesh, y, 0.2))
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - (k + 1)) < 0.15, (errs, rate)


def test_spatial_order_3d():
    errs = []
    for N in [2, 4, 8]:
        prob = Problem(3, N, 2, 3, 0.02)
        y = run_steps(prob, 2)
        errs.append(l2_error(prob.mesh, y, 0.04))
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - 3) < 0.3, (errs, rate)
