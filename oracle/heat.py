"""Manufactured heat problem u_t = Lap u + f on [0,1]^d, homogeneous Dirichlet (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in arXiv 2209.06700, Sec. 5: the heat equation is solved with a
manufactured solution on the unit cube, the source chosen to match, the
load integrated with the same (k+1)^d Gauss rule as the operators.  The
default workloads replace the paper's solution by
u = prod_a sin(pi x_a) cos t, so f = u_t - Lap u = S(x) (d pi^2 cos t - sin t)
with S = prod_a sin(pi x_a); S vanishes on the boundary (homogeneous
Dirichlet).  The weak form gives M y' + K y = g(t) with
g_j(t) = phi(t) G_j, G_j = int S phi_j, phi(t) = d pi^2 cos t - sin t.

Readings: the initial value is the nodal interpolant of u(., 0); the load
uses Gauss-Legendre (k+1)^d per cell (same rule as the matrices).

Pinned by tests: the load vector's quadrature rule by exact integration of a
degree-(2k+1) integrand against polynomial antiderivatives, its tensor-product
structure, and its entries against adaptive quadrature of int sin(pi x) phi_j
at the Gauss rule's rate (tests/test_oracle_heat_load.py); the spatial order
k+1 of the whole discretisation (tests/test_oracle_irk.py).
"""
import numpy as np

from .fem import Mesh, gauss_rule, gll_nodes, lagrange_values


def S_exact(x):
    """S(x) = prod_a sin(pi x_a); x has shape (..., d)."""
    return np.prod(np.sin(np.pi * x), axis=-1)


def phi_time(d, t):
    """Time factor of the source: f(x, t) = S(x) phi(t)."""
    return d * np.pi ** 2 * np.cos(t) - np.sin(t)


def u_exact(x, t):
    return S_exact(x) * np.cos(t)


def _cell_quadrature(mesh, npts):
    """Physical quadrature points (ncell, nq, d), weights (nq,) and basis values (nq, nb)."""
    d, N, k, p = mesh.d, mesh.N, mesh.k, mesh.p
    xq, wq = gauss_rule(npts)
    V, _ = lagrange_values(gll_nodes(k), xq)
    qidx = np.array(np.unravel_index(np.arange(npts ** d), (npts,) * d, order="F")).T
    bidx = np.array(np.unravel_index(np.arange(p ** d), (p,) * d, order="F")).T
    w = np.ones(npts ** d)
    phi = np.ones((npts ** d, p ** d))
    for a in range(d):
        w *= wq[qidx[:, a]]
        phi *= V[qidx[:, a]][:, bidx[:, a]]
    cells = np.array(np.unravel_index(np.arange(N ** d), (N,) * d, order="F")).T
    pts = (cells[:, None, :] + xq[qidx][None, :, :]) * mesh.h
    return pts, w * mesh.h ** d, phi


def load_vector(mesh):
    """G_j = int_Omega S phi_j by (k+1)^d-point Gauss per cell; zero on the boundary."""
    pts, w, phi = _cell_quadrature(mesh, mesh.p)
    Sq = S_exact(pts)                       # (ncell, nq)
    Ge = (Sq * w[None, :]) @ phi            # (ncell, nb)
    dofs = mesh.cell_dofs()
    G = np.bincount(dofs.reshape(-1), weights=Ge.reshape(-1), minlength=mesh.n)
    G[mesh.boundary_mask()] = 0.0
    return G


def initial_value(mesh, t=0.0):
    """Nodal interpolant of u(., t) (zero on the boundary)."""
    y = u_exact(mesh.node_coords(), t)
    y[mesh.boundary_mask()] = 0.0
    return y


def l2_error(mesh, y, t, extra=3):
    """|| u_h - u(t) ||_{L2(Omega)} with a (k+1+extra)-point Gauss rule per cell."""
    pts, w, phi = _cell_quadrature(mesh, mesh.p + extra)
    uh = y[mesh.cell_dofs()] @ phi.T        # (ncell, nq)
    err = uh - u_exact(pts, t)
    return float(np.sqrt(np.sum(err ** 2 * w[None, :])))
