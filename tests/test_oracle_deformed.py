"""Oracle pins for the heat problem on the curved mesh (CPU only).

Pins: eps = 0 reduces to the affine oracle; the Jacobian against finite differences of the map;
symmetry, definiteness, K 1 = 0 and the volume of the (unchanged) unit cube; the discrete energies
of the interpolant of S converge to the integrals of S^2 and |grad S|^2 (a transposed Jacobian or a
missing det J changes the limit); the heat solution converges at order k + 1 on the curved mesh;
the direct stage solve satisfies the stage system applied cell by cell.
"""
import numpy as np
import pytest

from oracle.deformed import (DeformedMesh, DeformedProblem, assemble_deformed, element_matrices_deformed,
                             initial_value_deformed, jacobian, l2_error_deformed, load_vector_deformed, phi_map)
from oracle.fem import Mesh, element_matrices, interior_restrict
from oracle.heat import initial_value, load_vector
from oracle.irk import apply_calA, step_direct


@pytest.mark.parametrize("d,N,k", [(2, 4, 2), (2, 3, 4), (3, 2, 3)])
def test_eps_zero_is_affine(d, N, k):
    m = DeformedMesh(d, N, k, 0.0)
    Me, Ke = element_matrices_deformed(m)
    Mr, Kr = element_matrices(d, k, 1.0 / N)
    assert np.abs(Me - Mr[None]).max() <= 1e-15 * np.abs(Mr).max()
    assert np.abs(Ke - Kr[None]).max() <= 1e-14 * np.abs(Kr).max()
    assert np.array_equal(load_vector_deformed(m), load_vector(Mesh(d, N, k)))
    assert np.array_equal(initial_value_deformed(m), initial_value(Mesh(d, N, k)))


@pytest.mark.parametrize("d", [2, 3])
def test_jacobian_finite_differences(d):
    rng = np.random.default_rng(0)
    xi = rng.uniform(0, 1, (20, d))
    eps, hh = 0.05, 1e-6
    J = jacobian(xi, eps)
    for b in range(d):
        e = np.zeros(d)
        e[b] = hh
        fd = (phi_map(xi + e, eps) - phi_map(xi - e, eps)) / (2 * hh)
        assert np.abs(J[:, :, b] - fd).max() < 1e-9


@pytest.mark.parametrize("d,N,k,eps", [(2, 4, 2, 0.1), (2, 3, 4, 0.1), (3, 2, 2, 0.05), (3, 3, 1, 0.05)])
def test_matrix_properties(d, N, k, eps):
    m = DeformedMesh(d, N, k, eps)
    M, K = assemble_deformed(m)
    assert abs(M - M.T).max() <= 1e-15 * abs(M).max()
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    assert np.abs(K @ np.ones(m.n)).max() <= 1e-13 * abs(K).max()
    assert abs(M.sum() - 1.0) <= 1e-13      # Phi maps the unit cube onto itself
    MI, _ = interior_restrict(m, M)
    KI, _ = interior_restrict(m, K)
    assert np.linalg.eigvalsh(MI.toarray()).min() > 0
    assert np.linalg.eigvalsh(KI.toarray()).min() > 0


@pytest.mark.parametrize("d,k,Ns,eps", [(2, 2, (4, 8, 16), 0.1), (2, 3, (4, 8, 16), 0.1), (3, 2, (2, 4, 8), 0.05)])
def test_energies_converge(d, k, Ns, eps):
    """u^T M u -> int S^2 = 2^-d and u^T K u -> int |grad S|^2 = d pi^2 2^-d, S at the mapped nodes."""
    errs = []
    for N in Ns:
        m = DeformedMesh(d, N, k, eps)
        M, K = assemble_deformed(m)
        S = np.prod(np.sin(np.pi * m.node_coords()), axis=-1)
        errs.append((abs(S @ (M @ S) - 0.5 ** d), abs(S @ (K @ S) - d * np.pi ** 2 * 0.5 ** d)))
    errs = np.array(errs)
    for j in range(2):
        assert errs[-1, j] < errs[-2, j] < errs[-3, j]
        assert errs[-2, j] / errs[-1, j] > 2 ** (k + 1)      # at least the L2 rate k+1
    assert errs[-1, 1] < (1e-4 if d == 2 else 1e-3)


def test_heat_spatial_order_deformed():
    k, errs = 2, []
    for N in [4, 8, 16]:
        prob = DeformedProblem(2, N, k, 3, 0.01, 0.1)
        y = prob.y0()
        for n in range(5):
            y = step_direct(prob, y, n * prob.tau)
        errs.append(l2_error_deformed(prob.mesh, y, 0.05))
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - (k + 1)) < 0.25, (errs, rate)


def test_direct_step_solves_stage_system():
    prob = DeformedProblem(3, 2, 3, 3, 0.01, 0.05)
    y = prob.y0()
    y1, kk = step_direct(prob, y, 0.0, return_stages=True)
    # (I (x) M + tau A (x) K) k = gbar - 1 (x) K y, applied cell by cell
    lhs = prob.apply_M(kk) + prob.tau * (prob.A @ prob.apply_K(kk))
    rhs = prob.stage_rhs_kron(y, 0.0)
    bmask = prob.mesh.boundary_mask()
    rhs[:, bmask] = 0.0
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()
    # Eq. (irk:A) form: calA k = (A^{-1} (x) I) rhs
    assert np.abs(apply_calA(prob, kk) - prob.Ainv @ rhs).max() <= 1e-11 * np.abs(rhs).max()
    assert np.abs(y1 - y).max() > 0


def test_cell_subset_matches_all_cells():
    m = DeformedMesh(3, 3, 2, 0.05)
    Me, Ke = element_matrices_deformed(m)
    sel = np.array([0, 5, 13, 26])
    Ms, Ks = element_matrices_deformed(m, cells=sel)
    assert np.array_equal(Ms, Me[sel]) and np.array_equal(Ks, Ke[sel])
