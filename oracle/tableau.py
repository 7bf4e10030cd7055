"""Radau IIA Butcher tableau and the small Q x Q factors of the method (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in arXiv 2209.06700:
* Sec. 1 (Introduction): y_{n+1} = y_n + tau sum_i b_i k_i with stage
  equations through A_Q = (a_ij), nodes c.
* Sec. 2, opening paragraph: Radau IIA with Q stages has order 2Q-1.  The
  paper does not print the coefficients; they are the collocation method on
  the right Radau points, built here from the textbook definition:
  c_1 < ... < c_Q are the zeros of d^{Q-1}/dx^{Q-1} [x^{Q-1} (x-1)^Q]
  (so c_Q = 1), a_ij = int_0^{c_i} l_j(s) ds and b_j = int_0^1 l_j(s) ds with
  l_j the Lagrange polynomials on the nodes c.
* Sec. 2, Eq. (irk:Ainv): A_Q^{-1} = S Lambda S^{-1}, floor(Q/2) complex
  pairs and one real eigenvalue for odd Q.  ``real_jordan`` gives the real
  2x2-block form used by the directly diagonalised variant (Sec. 6,
  Eq. (complex:twobytwo)), with beta = Im(lambda) > 0.
* Sec. 2, Eq. (irk:P): A_Q^{-1} = L U with U unit-diagonal (Axelsson and
  Neytcheva); L = S~ Lambda~ S~^{-1} is real.  ``crout_lu`` and
  ``lu_preconditioner_factors``.  Readings: no pivoting (Crout); S~ is
  scaled to unit diagonal and ordered like diag(L), so S~ is unit lower
  triangular and S~^{-1} is its forward-substitution inverse.

Pinned by tests/test_oracle_tableau.py: closed-form Q=2 and Q=3 tableaux,
the simplifying conditions B(2Q) / C(Q), the Q=2 stability function at a
printed point, R(z) against the (Q-1, Q) Pade approximant's known value
structure, L U == A^{-1}, spectrum(L^{-1} A^{-1}) == 1, the eigenvalue count
of A^{-1}.
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np


def radau_poly_coeffs(Q):
    """Integer coefficients (ascending powers) of d^{Q-1}/dx^{Q-1}[x^{Q-1}(x-1)^Q]."""
    # x^{Q-1}(x-1)^Q = sum_m C(Q,m) (-1)^{Q-m} x^{m+Q-1}; differentiate Q-1 times.
    coeffs = []
    for m in range(Q + 1):
        coeffs.append(comb(Q, m) * (-1) ** (Q - m) * factorial(m + Q - 1) // factorial(m))
    return coeffs


def _eval_exact(coeffs, x):
    acc = Fraction(0)
    for cf in reversed(coeffs):
        acc = acc * x + cf
    return acc


def radau_nodes(Q, grid=4096, bits=80):
    """Nodes c_1..c_Q: exact rational bisection on the integer polynomial.

    The roots are isolated by sign changes on a uniform rational grid over
    (0, 1] and then bisected in exact rational arithmetic, so the returned
    float64 values are correctly rounded up to the final conversion.
    """
    if Q < 1:
        raise ValueError("Q >= 1")
    coeffs = radau_poly_coeffs(Q)
    roots = []
    prev_x = Fraction(0)
    prev_v = _eval_exact(coeffs, prev_x)
    if prev_v == 0:
        raise AssertionError("x = 0 is not a Radau IIA node")
    for i in range(1, grid + 1):
        x = Fraction(i, grid)
        v = _eval_exact(coeffs, x)
        if v == 0:
            roots.append(x)
        elif (v > 0) != (prev_v > 0) and prev_v != 0:
            lo, hi, vlo = prev_x, x, prev_v
            for _ in range(bits):
                mid = (lo + hi) / 2
                vm = _eval_exact(coeffs, mid)
                if vm == 0:
                    lo = hi = mid
                    break
                if (vm > 0) == (vlo > 0):
                    lo, vlo = mid, vm
                else:
                    hi = mid
            roots.append((lo + hi) / 2)
        prev_x, prev_v = x, v
    if len(roots) != Q:
        raise AssertionError(f"found {len(roots)} Radau nodes for Q={Q}")
    return np.array([float(r) for r in roots])


def _lagrange(nodes, j, s):
    """l_j(s) on the given nodes, product form."""
    out = np.ones_like(s, dtype=np.float64)
    for m, cm in enumerate(nodes):
        if m != j:
            out = out * (s - cm) / (nodes[j] - cm)
    return out


def radau_iia(Q):
    """Return (A, b, c) of the Q-stage Radau IIA method (float64)."""
    c = radau_nodes(Q)
    # Gauss-Legendre with Q points integrates the degree Q-1 polynomials exactly.
    xg, wg = np.polynomial.legendre.leggauss(Q)
    A = np.zeros((Q, Q))
    b = np.zeros(Q)
    for i in range(Q):
        s = 0.5 * c[i] * (xg + 1.0)
        w = 0.5 * c[i] * wg
        for j in range(Q):
            A[i, j] = np.sum(w * _lagrange(c, j, s))
    s = 0.5 * (xg + 1.0)
    w = 0.5 * wg
    for j in range(Q):
        b[j] = np.sum(w * _lagrange(c, j, s))
    return A, b, c


def stability_function(A, b, z):
    """R(z) = 1 + z b^T (I - z A)^{-1} 1 (scalar test equation y' = lambda y, z = tau lambda)."""
    Q = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(Q) - z * A, np.ones(Q))


def crout_lu(Ainv):
    """Crout factorisation Ainv = L U, U unit upper triangular, no pivoting (Eq. irk:P)."""
    n = Ainv.shape[0]
    L = np.zeros((n, n))
    U = np.eye(n)
    for j in range(n):
        for i in range(j, n):
            L[i, j] = Ainv[i, j] - sum(L[i, m] * U[m, j] for m in range(j))
        if L[j, j] == 0.0:
            raise ZeroDivisionError("zero pivot in Crout LU")
        for i in range(j + 1, n):
            U[j, i] = (Ainv[j, i] - sum(L[j, m] * U[m, i] for m in range(j))) / L[j, j]
    return L, U


def lower_triangular_eigvecs(L):
    """Eigenvectors of lower-triangular L, column i for eigenvalue L[i,i], unit diagonal."""
    n = L.shape[0]
    S = np.zeros((n, n))
    for i in range(n):
        lam = L[i, i]
        S[i, i] = 1.0
        for m in range(i + 1, n):
            S[m, i] = sum(L[m, l] * S[l, i] for l in range(i, m)) / (lam - L[m, m])
    return S


def unit_lower_inverse(S):
    """Inverse of a unit lower-triangular matrix by forward substitution (column by column)."""
    n = S.shape[0]
    X = np.zeros((n, n))
    for j in range(n):
        X[j, j] = 1.0
        for i in range(j + 1, n):
            X[i, j] = -sum(S[i, l] * X[l, j] for l in range(j, i))
    return X


def lu_preconditioner_factors(Q):
    """Factors of Eq. (irk:P): returns dict with A, b, c, Ainv, L, U, lam (=diag L), S, Sinv."""
    A, b, c = radau_iia(Q)
    Ainv = np.linalg.inv(A)
    L, U = crout_lu(Ainv)
    S = lower_triangular_eigvecs(L)
    Sinv = unit_lower_inverse(S)
    return dict(A=A, b=b, c=c, Ainv=Ainv, L=L, U=U, lam=np.diag(L).copy(), S=S, Sinv=Sinv)


def real_jordan(Ainv):
    """Real block-diagonal form Ainv = T J T^{-1} (Eq. irk:Ainv in real arithmetic).

    Blocks, in order: one 1x1 block gamma for odd Q (real eigenvalue), then one
    2x2 block [[alpha, -beta], [beta, alpha]] per complex pair, beta > 0, so
    that (J (x) M + tau I (x) K) has the 2x2 form of Eq. (complex:twobytwo)
    with M' = beta M.  Returns (T, Tinv, blocks) with blocks a list of
    ('real', gamma) or ('pair', alpha, beta).
    """
    Q = Ainv.shape[0]
    w, V = np.linalg.eig(Ainv)
    real_idx = [i for i in range(Q) if abs(w[i].imag) < 1e-12 * abs(w[i])]
    pair_idx = [i for i in range(Q) if w[i].imag > 1e-12 * abs(w[i])]
    pair_idx.sort(key=lambda i: w[i].real)
    cols, blocks = [], []
    for i in real_idx:
        v = V[:, i].real
        cols.append(v)
        blocks.append(("real", w[i].real))
    for i in pair_idx:
        v = V[:, i]
        cols.append(v.real)
        cols.append(-v.imag)
        blocks.append(("pair", w[i].real, w[i].imag))
    T = np.array(cols).T
    if T.shape != (Q, Q):
        raise AssertionError("unexpected eigenstructure of A^{-1}")
    return T, np.linalg.inv(T), blocks


def block_matrix_J(blocks):
    """Assemble J from the block list of ``real_jordan``."""
    n = sum(1 if b[0] == "real" else 2 for b in blocks)
    J = np.zeros((n, n))
    o = 0
    for blk in blocks:
        if blk[0] == "real":
            J[o, o] = blk[1]
            o += 1
        else:
            _, al, be = blk
            J[o:o + 2, o:o + 2] = [[al, -be], [be, al]]
            o += 2
    return J
