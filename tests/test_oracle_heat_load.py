"""Pins of the oracle's load vector G_j = int S phi_j (Sec. 5: the load is integrated with the
same (k+1)^d Gauss rule as the element matrices).

Independent of the oracle's own basis and quadrature code:
* the rule: with the source replaced by a polynomial of degree k + 1 per axis, every integrand
  S phi_j has degree 2k + 1 per axis, which (k+1)-point Gauss integrates exactly and the
  (k+1)-point Gauss-Lobatto or a k-point Gauss rule do not; the exact integrals come from
  numpy's polynomial antiderivatives of Lagrange polynomials built by scipy on the textbook GLL
  nodes of tests/golden/gll_nodes_closed_forms.txt;
* the tensor structure: for the built-in S = prod sin(pi x_a) the 2D and 3D vectors are the outer
  products of the 1D one (a transposed or mixed index breaks this);
* the source itself: the 1D entries against int sin(pi x) phi_j by adaptive quadrature (scipy);
  the Gauss rule's relative error per entry falls like h^(k+2) (the first Taylor term of the sine
  it misses has degree k + 2 in the cell coordinate), a rule exact only to degree 2k - 1 like h^k.
"""
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.interpolate import lagrange

import oracle.heat as heat
from oracle.fem import Mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_nodes_closed_forms.txt")


def golden_gll(k):
    """GLL nodes on [0, 1] from the textbook closed forms (k = 1: the cell's end points)."""
    if k == 1:
        return np.array([0.0, 1.0])
    from math import sqrt  # noqa: F401  (used by eval of the closed forms)
    for line in open(GOLDEN):
        if line.startswith(f"k{k} "):
            return np.array([eval(tok, {"sqrt": sqrt}) for tok in line.split()[1:]], dtype=float)
    raise KeyError(k)


def exact_1d_load(N, k, poly):
    """G1_i = int_0^1 poly(x) phi_i(x) dx, exactly (polynomial antiderivatives), boundary zeroed."""
    xi = golden_gll(k)
    h = 1.0 / N
    G = np.zeros(k * N + 1)
    for c in range(N):
        for r in range(k + 1):
            ell = lagrange(xi, np.eye(k + 1)[r])              # reference basis function r on [0, 1]
            # in the cell coordinate s = (x - c h) / h: h int_0^1 poly(c h + h s) ell(s) ds
            pc = np.polyval(poly, np.poly1d([h, c * h]))
            anti = np.polyint(np.polymul(pc, ell))
            G[c * k + r] += h * (np.polyval(anti, 1.0) - np.polyval(anti, 0.0))
    G[0] = G[-1] = 0.0
    return G


@pytest.mark.parametrize("d,N,k", [(1, 3, 1), (1, 4, 2), (2, 3, 3), (3, 2, 4), (2, 5, 2), (3, 3, 1)])
def test_load_rule_exact_on_degree_2k_plus_1(monkeypatch, d, N, k):
    rng = np.random.default_rng(7 + k)
    coeffs = rng.uniform(-1.0, 1.0, k + 2)                  # degree k + 1, numpy.poly1d order
    poly = np.poly1d(coeffs)
    monkeypatch.setattr(heat, "S_exact", lambda x: np.prod(np.polyval(coeffs, x), axis=-1))
    G = heat.load_vector(Mesh(d, N, k))
    G1 = exact_1d_load(N, k, poly)
    ref = G1
    for _ in range(d - 1):
        ref = np.kron(G1, ref)
    assert np.abs(G - ref).max() <= 1e-13 * np.abs(ref).max()


def test_degree_2k_plus_2_is_not_exact(monkeypatch):
    """Control: one degree more than the rule integrates exactly leaves a visible error."""
    k, N = 2, 3
    coeffs = np.array([1.0, 0.0, 0.0, 0.0])                  # x^3 times a degree-2 basis: degree 5
    coeffs = np.concatenate([[1.0], coeffs])                 # x^4: degree 6 = 2k + 2
    monkeypatch.setattr(heat, "S_exact", lambda x: np.prod(np.polyval(coeffs, x), axis=-1))
    G = heat.load_vector(Mesh(1, N, k))
    ref = exact_1d_load(N, k, np.poly1d(coeffs))
    assert np.abs(G - ref).max() > 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_sine_load_tensor_structure(k):
    N = 4
    G1 = heat.load_vector(Mesh(1, N, k))
    G2 = heat.load_vector(Mesh(2, N, k))
    G3 = heat.load_vector(Mesh(3, N, k))
    assert np.allclose(G2, np.kron(G1, G1), rtol=0, atol=1e-15)
    assert np.allclose(G3, np.kron(G1, np.kron(G1, G1)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sine_load_against_exact_integrals(k):
    """The 1D entries approach int sin(pi x) phi_i with relative error falling like h^(k+2)."""
    errs = []
    for N in (4, 8):
        xi = golden_gll(k)
        h = 1.0 / N
        G = heat.load_vector(Mesh(1, N, k))
        ref = np.zeros_like(G)
        for c in range(N):
            for r in range(k + 1):
                ell = lagrange(xi, np.eye(k + 1)[r])
                f = lambda x, c=c, ell=ell: np.sin(np.pi * x) * ell((x - c * h) / h)
                ref[c * k + r] += quad(f, c * h, (c + 1) * h, epsabs=1e-15, epsrel=1e-14)[0]
        ref[0] = ref[-1] = 0.0
        errs.append(np.abs(G - ref).max() / np.abs(ref).max())
    assert errs[0] < 1e-3
    rate = np.log2(errs[0] / errs[1])
    assert rate > k + 1.5, (errs, rate)
