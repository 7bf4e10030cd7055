"""Oracle pins for the Radau IIA tableau and the preconditioner factors (CPU only).

Pins come from outside the oracle: textbook closed forms (tests/golden/),
the simplifying order conditions, the Pade form of the stability function,
and the algebraic facts the paper states in Sec. 2 around Eq. (irk:Ainv)
and Eq. (irk:P).
"""
import math
import os

import numpy as np
import pytest

from oracle.tableau import (block_matrix_J, crout_lu, lu_preconditioner_factors, radau_iia,
                            real_jordan, stability_function)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    env = {"s6": math.sqrt(6.0), "sqrt": math.sqrt}
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, rest = line.split(None, 1)
        rows = [[eval(tok, {"__builtins__": {}}, env) for tok in row.split()] for row in rest.split(";")]
        out[key] = np.array(rows if len(rows) > 1 else rows[0], dtype=np.float64)
    return out


def test_q2_closed_form():
    g = _golden("radau_iia_closed_forms.txt")
    A, b, c = radau_iia(2)
    np.testing.assert_allclose(c, g["c2"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(A, g["A2"], rtol=0, atol=2e-15)
    np.testing.assert_allclose(b, g["b2"], rtol=0, atol=2e-15)


def test_q3_closed_form():
    g = _golden("radau_iia_closed_forms.txt")
    A, b, c = radau_iia(3)
    np.testing.assert_allclose(c, g["c3"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(A, g["A3"], rtol=0, atol=2e-15)
    np.testing.assert_allclose(b, g["b3"], rtol=0, atol=2e-15)


def test_q2_stability_value():
    g = _golden("radau_iia_closed_forms.txt")
    A, b, _ = radau_iia(2)
    assert abs(stability_function(A, b, -3.7) - g["R2(-3.7)"]) < 1e-15


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_order_conditions(Q):
    """B(2Q-1): sum b_i c_i^{m-1} = 1/m; C(Q): sum_j a_ij c_j^{m-1} = c_i^m / m."""
    A, b, c = radau_iia(Q)
    for m in range(1, 2 * Q):
        assert abs(b @ c ** (m - 1) - 1.0 / m) < 5e-14
    for m in range(1, Q + 1):
        np.testing.assert_allclose(A @ c ** (m - 1), c ** m / m, rtol=0, atol=5e-14)
    assert c[-1] == 1.0
    np.testing.assert_allclose(A[-1], b, rtol=0, atol=5e-15)  # stiffly accurate


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 6])
def test_eigenvalues_of_Ainv_are_pade_denominator_roots(Q):
    """det(I - zA) is the (Q-1, Q) Pade denominator of e^z, so eig(A^{-1}) are its roots."""
    A, _, _ = radau_iia(Q)
    coeffs = [math.factorial(2 * Q - 1 - j) * math.factorial(Q)
              / (math.factorial(2 * Q - 1) * math.factorial(j) * math.factorial(Q - j)) * (-1) ** j
              for j in range(Q + 1)]
    roots = np.roots(coeffs[::-1])
    ev = np.linalg.eigvals(np.linalg.inv(A))
    for r in roots:
        assert np.min(np.abs(ev - r)) < 1e-9 * abs(r)
    n_complex = np.sum(np.abs(ev.imag) > 1e-10)
    assert n_complex == 2 * (Q // 2)
    assert np.sum(np.abs(ev.imag) <= 1e-10) == Q % 2


@pytest.mark.parametrize("Q", [1, 2, 3, 4])
def test_stability_function_is_pade(Q):
    """R(z) - e^z = O(z^{2Q}) for small z (order 2Q-1)."""
    A, b, _ = radau_iia(Q)
    z1 = {1: -0.02, 2: -0.05, 3: -0.1, 4: -0.25}[Q]   # error stays far above rounding
    z2 = z1 / 2
    e1 = abs(stability_function(A, b, z1) - math.exp(z1))
    e2 = abs(stability_function(A, b, z2) - math.exp(z2))
    assert abs(math.log2(e1 / e2) - 2 * Q) < 0.25


def test_q2_lu_values():
    f = lu_preconditioner_factors(2)
    np.testing.assert_allclose(f["Ainv"], [[1.5, 0.5], [-4.5, 2.5]], atol=2e-15)
    np.testing.assert_allclose(f["L"], [[1.5, 0.0], [-4.5, 4.0]], atol=2e-15)
    np.testing.assert_allclose(f["U"], [[1.0, 1.0 / 3.0], [0.0, 1.0]], atol=2e-15)


@pytest.mark.parametrize("Q", [2, 3, 4, 5, 6, 7, 8, 9])
def test_lu_factor_properties(Q):
    """A^{-1} = L U, U unit diagonal => eig(L^{-1} A^{-1}) = 1; L's spectrum is real (Eq. irk:P)."""
    f = lu_preconditioner_factors(Q)
    L, U, S, Sinv = f["L"], f["U"], f["S"], f["Sinv"]
    scale = np.abs(f["Ainv"]).max()
    np.testing.assert_allclose(L @ U, f["Ainv"], atol=1e-12 * scale)
    assert np.allclose(np.diag(U), 1.0)
    assert np.allclose(np.triu(L, 1), 0.0) and np.allclose(np.tril(U, -1), 0.0)
    # L^{-1} A^{-1} = U is unit upper triangular, so all its eigenvalues are exactly one
    LinvA = np.linalg.solve(L, f["Ainv"])
    np.testing.assert_allclose(np.tril(LinvA, -1), 0.0, atol=1e-9)
    np.testing.assert_allclose(np.diag(LinvA), 1.0, atol=1e-9)
    np.testing.assert_allclose(L @ S, S @ np.diag(f["lam"]), atol=1e-10 * scale * np.abs(S).max())
    np.testing.assert_allclose(S @ Sinv, np.eye(Q), atol=1e-9)
    assert np.all(f["lam"] > 0)                   # every LU block lambda M + tau K is SPD
    assert abs(f["lam"][-1] - Q * Q) < 1e-9 * Q * Q  # observed L_QQ = Q^2


def test_crout_is_plain_lu_without_pivoting():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5, 5)) + 5 * np.eye(5)
    L, U = crout_lu(X)
    np.testing.assert_allclose(L @ U, X, atol=1e-13)


@pytest.mark.parametrize("Q", [2, 3, 4, 5])
def test_real_jordan(Q):
    A, _, _ = radau_iia(Q)
    Ainv = np.linalg.inv(A)
    T, Tinv, blocks = real_jordan(Ainv)
    J = block_matrix_J(blocks)
    np.testing.assert_allclose(T @ J @ Tinv, Ainv, atol=1e-12 * np.abs(Ainv).max())
    assert sum(1 for b in blocks if b[0] == "pair") == Q // 2
    assert all(b[2] > 0 for b in blocks if b[0] == "pair")


def test_q3_real_jordan_values():
    A, _, _ = radau_iia(3)
    _, _, blocks = real_jordan(np.linalg.inv(A))
    # roots of z^3 - 9 z^2 + 36 z - 60 (Pade (2,3) denominator, scaled)
    roots = np.roots([1.0, -9.0, 36.0, -60.0])
    gamma = roots[np.abs(roots.imag) < 1e-12].real[0]
    pair = roots[roots.imag > 1e-12][0]
    assert abs(blocks[0][1] - gamma) < 1e-12
    assert abs(blocks[1][1] - pair.real) < 1e-12 and abs(blocks[1][2] - pair.imag) < 1e-12


@pytest.mark.parametrize("Q", [3, 6, 9])
def test_sinv_against_extended_precision(Q):
    """S~^{-1} by forward substitution is accurate even at cond(S~) ~ 5e9 (Q = 9)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    f = lu_preconditioner_factors(Q)
    hp = np.array((mpmath.matrix(f["S"].tolist()) ** -1).tolist(), dtype=float)
    assert np.abs(f["Sinv"] - hp).max() <= 1e-13 * np.abs(hp).max()
    assert np.all(np.triu(f["Sinv"], 1) == 0.0)
