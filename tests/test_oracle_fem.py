"""Oracle pins for the Q_k finite-element matrices (CPU only).

Pins: closed-form GLL nodes (tests/golden/), exact integrals of polynomial
products (Gauss with k+1 points integrates degree 2k+1 exactly), symmetry
and definiteness, partition of unity, the Kronecker structure of M and K on
the uniform mesh, and agreement of the two apply routes.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import (Mesh, apply_cellwise, assemble, element_matrices, gll_nodes,
                        interior_restrict)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gll_golden():
    out = {}
    for line in open(os.path.join(GOLDEN, "gll_nodes_closed_forms.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            key, rest = line.split(None, 1)
            out[int(key[1:])] = np.array([eval(t, {"__builtins__": {}}, {"sqrt": math.sqrt})
                                          for t in rest.split()])
    return out


@pytest.mark.parametrize("k", [2, 3, 4])
def test_gll_nodes(k):
    np.testing.assert_allclose(gll_nodes(k), _gll_golden()[k], rtol=0, atol=2e-16 * 8)


@pytest.mark.parametrize("d,N,k", [(2, 3, 1), (2, 2, 3), (3, 2, 2)])
def test_matrix_properties(d, N, k):
    mesh = Mesh(d, N, k)
    M, K = assemble(mesh)
    assert abs(M - M.T).max() < 1e-15
    assert abs(K - K.T).max() < 1e-13
    assert abs(M.sum() - 1.0) < 1e-13                       # integral of 1 over the unit cube
    assert np.abs(K @ np.ones(mesh.n)).max() < 1e-12         # constants are in the kernel of K
    MI, _ = interior_restrict(mesh, M)
    KI, _ = interior_restrict(mesh, K)
    assert np.linalg.eigvalsh(MI.toarray()).min() > 0
    assert np.linalg.eigvalsh(KI.toarray()).min() > 0


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_polynomial_exactness_2d(k):
    mesh = Mesh(2, 3, k)
    M, K = assemble(mesh)
    X = mesh.node_coords()
    for (a, b, c, e) in [(k, 0, 1, k), (k, k, k, k), (1, 1, 0, 0)]:
        u = X[:, 0] ** a * X[:, 1] ** b
        v = X[:, 0] ** c * X[:, 1] ** e
        exact_m = 1.0 / ((a + c + 1) * (b + e + 1))
        assert abs(u @ (M @ v) - exact_m) < 1e-13
        # grad u . grad v integrated exactly (degree <= 2k per direction)
        # d/dx terms: a c int x^{a+c-2} int y^{b+e}; d/dy likewise
        gx = a * c / (a + c - 1) / (b + e + 1) if a > 0 and c > 0 else 0.0
        gy = b * e / (b + e - 1) / (a + c + 1) if b > 0 and e > 0 else 0.0
        assert abs(u @ (K @ v) - (gx + gy)) < 1e-12


@pytest.mark.parametrize("d,N,k", [(2, 4, 2), (3, 2, 3), (3, 3, 1)])
def test_cellwise_equals_csr(d, N, k):
    mesh = Mesh(d, N, k)
    M, K = assemble(mesh)
    Me, Ke = element_matrices(d, k, mesh.h)
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, mesh.n)
    bm = mesh.boundary_mask()
    u[bm] = 0.0
    for A, Ce in ((M, Me), (K, Ke)):
        ref = A @ u
        ref[bm] = 0.0
        got = apply_cellwise(mesh, Ce, u)
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max() * 10


@pytest.mark.parametrize("d,N,k", [(2, 3, 2), (3, 2, 2), (3, 2, 4)])
def test_kronecker_structure(d, N, k):
    """With Gauss (k+1)^d, M = M1 (x) .. (x) M1 and K = sum of K1 in one slot, exactly."""
    mesh = Mesh(d, N, k)
    M, K = assemble(mesh)
    M1, K1 = assemble(Mesh(1, N, k))
    M1, K1 = M1.toarray(), K1.toarray()

    def kron_list(mats):
        out = np.ones((1, 1))
        for m in mats:  # x fastest: last factor is x
            out = np.kron(out, m)
        return out

    Mk = kron_list([M1] * d)
    Kk = sum(kron_list([K1 if i == j else M1 for i in range(d)]) for j in range(d))
    assert np.abs(M.toarray() - Mk).max() < 1e-15
    assert np.abs(K.toarray() - Kk).max() < 1e-12
