"""Oracle pins for the multigrid, Chebyshev and PRESB ingredients (CPU only).

Pins: the Chebyshev error-propagation polynomial in closed form; exact
reproduction of Q_k polynomials by the prolongation; V-cycle symmetry and
contraction; the PRESB factorisation of Eq. (presb:p) and its spectral
bound [1/2, 1].
"""
import numpy as np
import pytest

from oracle.fem import Mesh
from oracle.mg import (VCycle, chebyshev, jacobi_diag, level_operator, level_sizes, presb_apply,
                       presb_factors, prolongation)


def test_level_sizes():
    assert level_sizes(32, 4) == [32, 16, 8, 4, 2, 1]
    assert level_sizes(48, 2) == [48, 24, 12, 6, 3]
    assert level_sizes(16, 1) == [16, 8, 4, 2]
    assert level_sizes(64, 3) == [64, 32, 16, 8, 4, 2, 1]


def test_chebyshev_error_polynomial():
    """e_m = T_m((theta - mu)/delta) / T_m(theta/delta) e_0 on every eigenpair of D^{-1}A."""
    A, bm = level_operator(2, 3, 2, 2.0, 0.05)
    D = jacobi_diag(A, bm)
    keep = ~bm
    s = 1.0 / np.sqrt(D[keep])
    mu, W = np.linalg.eigh(s[:, None] * A[np.ix_(keep, keep)] * s[None, :])
    lo, hi = 0.3 * mu.max(), 1.1 * mu.max()
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    x_true = np.zeros(A.shape[0])
    for m in (1, 2, 3, 5):
        for idx in (0, len(mu) // 2, len(mu) - 1):
            # eigenvector of D^{-1}A: v = D^{-1/2} w
            v = np.zeros(A.shape[0])
            v[keep] = s * W[:, idx]
            x0 = v.copy()                      # error e_0 = x0 - x_true = v (b = 0)
            x = chebyshev(A, D, A @ x_true, x0, m, lo, hi, bm)
            T = np.polynomial.chebyshev.Chebyshev.basis(m)
            factor = T((theta - mu[idx]) / delta) / T(theta / delta)
            np.testing.assert_allclose(x, factor * v, atol=1e-12 * np.abs(v).max())


@pytest.mark.parametrize("d,Nc,k", [(2, 2, 1), (2, 2, 3), (3, 1, 2), (3, 2, 2), (2, 3, 4)])
def test_prolongation_reproduces_polynomials(d, Nc, k):
    P = prolongation(d, Nc, k)
    mc, mf = Mesh(d, Nc, k), Mesh(d, 2 * Nc, k)
    xc, xf = mc.node_coords(), mf.node_coords()
    # a Q_k polynomial that vanishes on the boundary (Dirichlet) of degree k per direction
    def f(x):
        out = np.ones(len(x))
        for a in range(d):
            out *= x[:, a] * (1 - x[:, a]) * (x[:, a] + 0.3) ** (k - 2) if k >= 2 else x[:, a] * 0 + 1
        return out
    if k == 1:
        # piecewise-linear hat functions: check the coarse interpolant of a hat is reproduced
        uc = np.zeros(mc.n)
        uc[~mc.boundary_mask()] = np.arange(1, np.sum(~mc.boundary_mask()) + 1)
        uf = P @ uc
        assert np.all(np.isfinite(uf))
        return
    np.testing.assert_allclose(P @ f(xc), f(xf), atol=1e-14)


def test_prolongation_is_interpolation_at_shared_nodes():
    P = prolongation(2, 2, 2)
    mc, mf = Mesh(2, 2, 2), Mesh(2, 4, 2)
    xc, xf = mc.node_coords(), mf.node_coords()
    for ic in np.flatnonzero(~mc.boundary_mask()):
        jf = np.flatnonzero(np.all(np.abs(xf - xc[ic]) < 1e-14, axis=1))[0]
        row = P[jf]
        assert abs(row[ic] - 1.0) < 1e-14 and abs(row.sum() - 1.0) < 1e-14


def test_vcycle_symmetric_and_contracting():
    V = VCycle(2, 8, 2, 3.0, 0.01, 3)
    A, bm = V.levels[0]["A"], V.levels[0]["bm"]
    rng = np.random.default_rng(0)
    x = rng.standard_normal(A.shape[0])
    y = rng.standard_normal(A.shape[0])
    x[bm] = y[bm] = 0.0
    Bx, By = V.apply(x), V.apply(y)
    assert abs(x @ By - y @ Bx) < 1e-12 * abs(x @ Bx)
    assert x @ Bx > 0
    keep = ~bm
    B = np.array([V.apply(e) for e in np.eye(A.shape[0])]).T
    E = np.eye(A.shape[0]) - B @ A
    rho = max(abs(np.linalg.eigvals(E[np.ix_(keep, keep)])))
    assert rho < 0.5


def test_presb_factorisation_and_bound():
    rng = np.random.default_rng(2)
    n = 6
    X = rng.standard_normal((n, n))
    M = X @ X.T + n * np.eye(n)
    Y = rng.standard_normal((n, n))
    K = Y @ Y.T + 0.1 * np.eye(n)
    alpha, beta, tau = 2.68, 3.05, 0.01
    Kp, Mp = alpha * M + tau * K, beta * M
    Xf, Yf, Zf, P = presb_factors(Kp, Mp)
    np.testing.assert_allclose(Xf @ Yf @ Zf, P, atol=1e-12 * np.abs(P).max())
    A2 = np.block([[Kp, -Mp], [Mp, Kp]])
    ev = np.linalg.eigvals(np.linalg.solve(P, A2))
    assert ev.real.min() > 0.5 - 1e-10 and ev.real.max() < 1.0 + 1e-10
    H = Kp + Mp
    f, g = rng.standard_normal(n), rng.standard_normal(n)
    u, v = presb_apply(lambda r: np.linalg.solve(H, r), lambda w: Mp @ w, f, g)
    np.testing.assert_allclose(P @ np.concatenate([u, v]), np.concatenate([f, g]), atol=1e-11)


# ---- the coupled 2x2 V-cycle (Sec. 6, GMG applied directly to Eq. complex:twobytwo)

def _bounds(d, N, k, lam, tau):
    from oracle.mg import max_eig_DinvA
    out = []
    for Nl in level_sizes(N, k):
        A, bm = level_operator(d, Nl, k, lam, tau)
        hi = 1.2 * max_eig_DinvA(A, jacobi_diag(A, bm), bm)
        out.append((hi / 20.0, hi))
    return out


def test_coupled_vcycle_without_coupling_is_two_scalar_vcycles():
    from oracle.mg import CoupledVCycle, VCycle
    d, N, k, alpha, tau = 2, 8, 2, 2.7, 1e-2
    bounds = _bounds(d, N, k, alpha, tau)
    cv = CoupledVCycle(d, N, k, alpha, 0.0, tau, 3, bounds)
    sv = VCycle(d, N, k, alpha, tau, 3, bounds=bounds)
    rng = np.random.default_rng(3)
    n = (k * N + 1) ** d
    b = rng.uniform(-1, 1, 2 * n)
    b[np.concatenate([cv.levels[0]["bm"][:n]] * 2)] = 0.0
    got = cv.apply(b)
    ref = np.concatenate([sv.apply(b[:n]), sv.apply(b[n:])])
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_coupled_nodal_jacobi_inverts_the_nodal_blocks():
    from oracle.mg import coupled_level
    d, N, k = 2, 4, 3
    C, dinv, bm = coupled_level(d, N, k, 2.0, 3.0, 1e-2)
    n = C.shape[0] // 2
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, 2 * n)
    z[bm] = 0.0
    # nodal blocks of C: [[C[i,i], C[i,n+i]], [C[n+i,i], C[n+i,n+i]]]
    i = np.arange(n)
    r0 = C[i, i] * z[:n] + C[i, n + i] * z[n:]
    r1 = C[n + i, i] * z[:n] + C[n + i, n + i] * z[n:]
    r = np.concatenate([r0, r1])
    r[bm] = 0.0
    assert np.abs(dinv(r) - z).max() <= 1e-12 * np.abs(z).max()


def test_coupled_vcycle_contracts_the_error():
    from oracle.mg import CoupledVCycle
    d, N, k, alpha, beta, tau = 2, 8, 2, 2.68, 3.05, 1e-3
    cv = CoupledVCycle(d, N, k, alpha, beta, tau, 3, _bounds(d, N, k, alpha, tau))
    A, bm = cv.levels[0]["A"], cv.levels[0]["bm"]
    rng = np.random.default_rng(5)
    e = rng.uniform(-1, 1, A.shape[0])
    e[bm] = 0.0
    e0 = np.linalg.norm(e)
    for _ in range(5):  # e <- (I - B A) e
        e = e - cv.apply(A @ e)
    assert np.linalg.norm(e) <= 0.5 ** 5 * e0


@pytest.mark.parametrize("d,Nc,k", [(2, 2, 1), (2, 3, 3), (3, 2, 2), (3, 1, 4), (3, 3, 1)])
def test_sparse_forms_equal_the_dense_definitions(d, Nc, k):
    """The sparse prolongation (Kronecker product of 1D embeddings) and the sparse level operator
    equal the dense ones built from their definitions (coarse basis at each fine node; assembled
    lambda M + tau K with boundary rows and columns zeroed)."""
    from oracle.mg import level_operator_sparse, prolongation_sparse
    Pd = prolongation(d, Nc, k)
    Ps = prolongation_sparse(d, Nc, k).toarray()
    assert np.abs(Pd - Ps).max() <= 1e-15
    A, bm = level_operator(d, 2 * Nc, k, 1.7, 0.3)
    As, bs = level_operator_sparse(d, 2 * Nc, k, 1.7, 0.3)
    assert np.array_equal(bm, bs)
    assert np.abs(A - As.toarray()).max() <= 1e-15 * np.abs(A).max()
    assert np.array_equal(jacobi_diag(A, bm), jacobi_diag(As, bs))
