"""The library's host-built 1D Q_k element data (irk_element_factors: what every operator launch
takes as coefficients) against the oracle's (CPU, no device): GLL nodes, the Gauss rule, the
reference mass and stiffness matrices, basis values and derivatives at the Gauss points, and the
prolongation block of a split cell (the coarse basis evaluated at the fine mesh's nodes)."""
import ctypes

import numpy as np
import pytest

from oracle.fem import Mesh, element_matrices, gauss_rule, gll_nodes, lagrange_values


@pytest.fixture(scope="module")
def pkg():
    from tests.test_capi_load import _built_lib
    _built_lib()
    import paper_2209_06700_gb300 as p
    return p


def _close(got, ref, tol):
    assert got.shape == np.shape(ref)
    assert np.abs(got - ref).max() <= tol * max(np.abs(ref).max(), 1.0), np.abs(got - ref).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_element_data_matches_the_oracle(pkg, k):
    nodes = gll_nodes(k)
    gq, gw = gauss_rule(k + 1)
    V, D = lagrange_values(nodes, gq)
    Me, Ke = element_matrices(1, k, 1.0)
    _close(pkg.element_factors(k, "nodes"), nodes, 1e-15)
    # the order of the Gauss points is free (every use sums over them): compare sorted by point
    order = np.argsort(pkg.element_factors(k, "gq"))
    _close(pkg.element_factors(k, "gq")[order], gq, 1e-15)
    _close(pkg.element_factors(k, "gw")[order], gw, 1e-15)
    _close(pkg.element_factors(k, "B")[order], V, 1e-14)
    _close(pkg.element_factors(k, "D")[order], D, 1e-13)
    _close(pkg.element_factors(k, "Me"), Me, 1e-15)
    _close(pkg.element_factors(k, "Ke"), Ke, 1e-13)
    # the coarse cell [0, 1] split in two: fine nodes of the 2-cell mesh of the same degree
    xf = Mesh(1, 2, k).node_coords()[:, 0]
    Pf, _ = lagrange_values(nodes, xf)
    _close(pkg.element_factors(k, "Pc"), Pf, 1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_element_data_invariants(pkg, k):
    """Partition of unity of the basis (rows of B and Pc sum to 1, rows of D to 0), the mass
    matrix integrates 1 (sum = cell length), the stiffness matrix annihilates constants."""
    B, D, Pc = (pkg.element_factors(k, n) for n in ("B", "D", "Pc"))
    Me, Ke = pkg.element_factors(k, "Me"), pkg.element_factors(k, "Ke")
    assert np.abs(B.sum(axis=1) - 1).max() < 1e-14 and np.abs(Pc.sum(axis=1) - 1).max() < 1e-14
    assert np.abs(D.sum(axis=1)).max() < 1e-12
    assert abs(Me.sum() - 1.0) < 1e-14 and np.abs(Ke @ np.ones(k + 1)).max() < 1e-12


def test_invalid_arguments_are_refused(pkg):
    from paper_2209_06700_gb300 import _capi
    lib = pkg.lib()
    out = (ctypes.c_double * 64)()
    assert lib.irk_element_factors(0, 0, out) == _capi.IRK_EINVAL
    assert lib.irk_element_factors(5, 0, out) == _capi.IRK_EINVAL
    assert lib.irk_element_factors(2, 8, out) == _capi.IRK_EINVAL
    assert lib.irk_element_factors(2, 0, None) == _capi.IRK_EINVAL
