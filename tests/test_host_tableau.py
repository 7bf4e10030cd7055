"""Step a1 of the product on the host (CPU, no device): the library's Radau IIA tableau and its
factors (irk_tableau_factors, built by the routine irk_create uses) against the oracle's
(oracle/tableau.py: exact rational bisection for the nodes, Gauss quadrature for A, Crout LU,
substitution for the eigenvectors of L).  The two share no code."""
import ctypes

import numpy as np
import pytest

from oracle.tableau import lu_preconditioner_factors, radau_iia, real_jordan


@pytest.fixture(scope="module")
def pkg():
    from tests.test_capi_load import _built_lib
    _built_lib()
    import paper_2209_06700_gb300 as p
    return p


def _close(got, ref, rtol):
    scale = max(np.abs(ref).max(), 1e-300)
    assert got.shape == np.shape(ref)
    assert np.abs(got - ref).max() <= rtol * scale, (np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("Q", range(1, 10))
def test_tableau_and_lu_factors_match_the_oracle(pkg, Q):
    A, b, c = radau_iia(Q)
    _close(pkg.tableau_factors(Q, "A"), A, 1e-14)
    _close(pkg.tableau_factors(Q, "b"), b, 1e-14)
    _close(pkg.tableau_factors(Q, "c"), c, 1e-14)
    if Q == 1:
        return
    f = lu_preconditioner_factors(Q)
    cond = np.linalg.cond(f["S"])
    _close(pkg.tableau_factors(Q, "Ainv"), f["Ainv"], 1e-13)
    _close(pkg.tableau_factors(Q, "L"), f["L"], 1e-13)
    _close(pkg.tableau_factors(Q, "U"), f["U"], 1e-13)
    _close(pkg.tableau_factors(Q, "lam"), f["lam"], 1e-13)
    # S~ is unit lower triangular with columns ordered like diag(L): unique, conditioned by cond(S~)
    _close(pkg.tableau_factors(Q, "S"), f["S"], 1e-15 * cond)
    _close(pkg.tableau_factors(Q, "Sinv"), f["Sinv"], 1e-15 * cond)


@pytest.mark.parametrize("Q", range(2, 10))
def test_real_block_form_matches_the_oracle(pkg, Q):
    """T is not unique: check T J T^{-1} = A^{-1} and the block values (gamma, alpha +- i beta,
    beta > 0) against the oracle's real Jordan form."""
    Ainv = pkg.tableau_factors(Q, "Ainv")
    T, Tinv, J = (pkg.tableau_factors(Q, n) for n in ("T", "Tinv", "J"))
    _close(T @ J @ Tinv, Ainv, 1e-11)
    _close(T @ Tinv, np.eye(Q), 1e-11)
    _, _, blocks = real_jordan(np.linalg.inv(radau_iia(Q)[0]))
    ref = sorted((round(blk[1], 9), round(blk[2], 9) if blk[0] == "pair" else 0.0) for blk in blocks)
    got, i = [], 0
    while i < Q:   # walk the block diagonal of J: 1x1 real blocks, 2x2 [[a, -b], [b, a]] pairs
        if i + 1 < Q and abs(J[i + 1, i]) > 0:
            assert J[i, i] == J[i + 1, i + 1] and J[i, i + 1] == -J[i + 1, i] and J[i + 1, i] > 0
            got.append((round(J[i, i], 9), round(J[i + 1, i], 9)))
            i += 2
        else:
            got.append((round(J[i, i], 9), 0.0))
            i += 1
    assert sorted(got) == ref


def test_invalid_arguments_are_refused(pkg):
    from paper_2209_06700_gb300 import _capi
    lib = pkg.lib()
    out = (ctypes.c_double * 81)()
    assert lib.irk_tableau_factors(0, 0, out) == _capi.IRK_EINVAL
    assert lib.irk_tableau_factors(10, 0, out) == _capi.IRK_EINVAL
    assert lib.irk_tableau_factors(3, 12, out) == _capi.IRK_EINVAL
    assert lib.irk_tableau_factors(3, 0, None) == _capi.IRK_EINVAL
