"""The paper's own manufactured heat problem (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in arXiv 2209.06700, Sec. 5 (experimental setup): the 3D heat equation
on the unit cube with the analytic solution
    u(x, t) = prod_a sin(2 pi x_a) (1 + sin(pi t)) exp(-t/2),
homogeneous Dirichlet data, Q_k elements with Gauss (k+1)^d quadrature,
tau = 0.1.  The source follows from u_t - Lap u: with S2 = prod_a sin(2 pi x_a)
(-Lap S2 = 4 d pi^2 S2) and theta(t) = (1 + sin pi t) e^{-t/2},
    f(x, t) = S2(x) (theta'(t) + 4 d pi^2 theta(t)),
    theta'(t) = (pi cos pi t - (1 + sin pi t) / 2) e^{-t/2},
so the semi-discrete load is g(t) = psi(t) G2 with G2_j = int S2 phi_j and
psi = theta' + 4 d pi^2 theta.  The initial value is the nodal interpolant
of u(., 0) = S2.

Pinned by tests/test_oracle_paper_workload.py: spatial order k+1 of the
whole discretisation against this u, and agreement of the fast-diagonalised
step with the sparse direct Kronecker solve on these loads.
"""
import numpy as np

from .heat import _cell_quadrature


def S2(x):
    """prod_a sin(2 pi x_a); x has shape (..., d)."""
    return np.prod(np.sin(2.0 * np.pi * x), axis=-1)


def theta(t):
    return (1.0 + np.sin(np.pi * t)) * np.exp(-0.5 * t)


def theta_prime(t):
    return (np.pi * np.cos(np.pi * t) - 0.5 * (1.0 + np.sin(np.pi * t))) * np.exp(-0.5 * t)


def psi(d, t):
    """Time factor of the load: f(x, t) = S2(x) psi(t)."""
    return theta_prime(t) + 4.0 * d * np.pi ** 2 * theta(t)


def u_exact(x, t):
    return S2(x) * theta(t)


def load_vector(mesh):
    """G2_j = int S2 phi_j by (k+1)^d-point Gauss per cell; zero on the boundary."""
    pts, w, phi = _cell_quadrature(mesh, mesh.p)
    Ge = (S2(pts) * w[None, :]) @ phi
    dofs = mesh.cell_dofs()
    G = np.bincount(dofs.reshape(-1), weights=Ge.reshape(-1), minlength=mesh.n)
    G[mesh.boundary_mask()] = 0.0
    return G


def initial_value(mesh):
    y = S2(mesh.node_coords())
    y[mesh.boundary_mask()] = 0.0
    return y


def stage_loads(prob, G2, t_n):
    """(Q, n): g(t_n + c_i tau) = psi(t_n + c_i tau) G2."""
    return np.stack([psi(prob.d, t_n + ci * prob.tau) * G2 for ci in prob.c])


def l2_error(mesh, y, t, extra=3):
    """|| u_h - u(t) ||_{L2} with a (k+1+extra)-point Gauss rule per cell."""
    pts, w, phi = _cell_quadrature(mesh, mesh.p + extra)
    uh = y[mesh.cell_dofs()] @ phi.T
    err = uh - u_exact(pts, t)
    return float(np.sqrt(np.sum(err ** 2 * w[None, :])))
