"""The heat problem of oracle.heat on a curved (non-affine) mesh of [0,1]^d (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Source in arXiv 2209.06700, Sec. 3.4 (batching of operations): on deformed cells a
matrix-free loop loads the mapping data, the Jacobian of the cell map at every
quadrature point, and batching all Q stages into one cell loop loads it once
instead of Q times.  The paper itself runs affine meshes only and prints no
deformed mesh, so this module fixes one (reading):

* the uniform mesh of oracle.fem mapped by Phi(xi) = xi + eps S(xi) (1, .., 1),
  S = prod_a sin(pi xi_a): Phi fixes the boundary of the cube, is non-affine in
  every cell, and is one-to-one for eps d pi < 1 (det J = 1 + eps sum_a dS/dxi_a);
* the geometry enters only through J = dPhi/dxi at the quadrature points (the
  exact map, no isoparametric approximation); cell integrals use the same
  Gauss-Legendre (k+1)^d rule as the affine case:
      M_e[i, j] = sum_q w_q det J_q phi_i phi_j,
      K_e[i, j] = sum_q w_q det J_q (J_q^-T grad phi_i) . (J_q^-T grad phi_j);
* the manufactured solution u = S(x) cos t is taken in physical coordinates
  x = Phi(xi), so the source f = S(x) (d pi^2 cos t - sin t) and the initial
  value (the interpolant at the mapped nodes) are those of oracle.heat.

Everything is direct quadrature with dense per-cell matrices (no sum
factorisation).  Pinned by tests/test_oracle_deformed.py: eps = 0 gives the
affine matrices, load and initial value exactly; M and K symmetric, M positive
definite, K 1 = 0; sum(M) -> 1 (the mapped domain is still the unit cube); the
discrete energies u^T M u and u^T K u of the interpolant of S converge to the
integrals of S^2 and |grad S|^2 over the cube; the heat solution converges at
order k + 1 in L2 on the curved mesh.
"""
import numpy as np
import scipy.sparse as sp

from .fem import Mesh, gauss_rule, gll_nodes, lagrange_values
from .heat import S_exact, phi_time, u_exact
from .tableau import radau_iia


def phi_map(xi, eps):
    """Phi(xi) = xi + eps S(xi) 1; xi has shape (..., d)."""
    return xi + eps * S_exact(xi)[..., None]


def jacobian(xi, eps):
    """J[..., a, b] = dPhi_a / dxi_b = delta_ab + eps dS/dxi_b."""
    d = xi.shape[-1]
    s = np.sin(np.pi * xi)
    c = np.cos(np.pi * xi)
    grad = np.empty(xi.shape)
    for b in range(d):
        g = np.pi * c[..., b]
        for a in range(d):
            if a != b:
                g = g * s[..., a]
        grad[..., b] = g
    J = np.broadcast_to(np.eye(d), xi.shape[:-1] + (d, d)).copy()
    J += eps * grad[..., None, :]
    return J


class DeformedMesh(Mesh):
    """Mesh(d, N, k) whose cells are mapped by Phi with amplitude eps."""

    def __init__(self, d, N, k, eps):
        super().__init__(d, N, k)
        if eps * d * np.pi >= 1.0:
            raise ValueError("eps d pi < 1 keeps the map one-to-one")
        self.eps = float(eps)

    def node_coords(self):
        """Physical node coordinates Phi(xi_node), (n, d)."""
        return phi_map(super().node_coords(), self.eps)

    def quadrature(self, npts=None, cells=None):
        """Reference points xi (ncell, nq, d), weights w_q h^d (nq,), basis values (nq, nb) and
        reference gradients (nq, nb, d) in the cell coordinate xi (not the unit-cell one); for the
        listed cell indices only (x fastest) when ``cells`` is given."""
        d, N, k, p, h = self.d, self.N, self.k, self.p, self.h
        npts = p if npts is None else npts
        xq, wq = gauss_rule(npts)
        V, D = lagrange_values(gll_nodes(k), xq)
        qidx = np.array(np.unravel_index(np.arange(npts ** d), (npts,) * d, order="F")).T
        bidx = np.array(np.unravel_index(np.arange(p ** d), (p,) * d, order="F")).T
        w = np.ones(npts ** d)
        phi = np.ones((npts ** d, p ** d))
        grad = np.ones((npts ** d, p ** d, d))
        for a in range(d):
            w *= wq[qidx[:, a]]
            Va = V[qidx[:, a]][:, bidx[:, a]]
            Da = D[qidx[:, a]][:, bidx[:, a]] / h
            phi *= Va
            for g in range(d):
                grad[:, :, g] *= Da if g == a else Va
        ids = np.arange(N ** d) if cells is None else np.asarray(cells)
        cidx = np.array(np.unravel_index(ids, (N,) * d, order="F")).T
        xi = (cidx[:, None, :] + xq[qidx][None, :, :]) * h
        return xi, w * h ** d, phi, grad


def element_matrices_deformed(mesh, cells=None):
    """Per-cell dense mass and stiffness matrices (ncell, nb, nb) by direct quadrature (all cells,
    or the listed cell indices)."""
    xi, w, phi, grad = mesh.quadrature(cells=cells)
    J = jacobian(xi, mesh.eps)                      # (ncell, nq, d, d)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    wdet = w[None, :] * det                         # (ncell, nq)
    Me = np.einsum("cq,qi,qj->cij", wdet, phi, phi)
    # physical gradients: grad_x phi = J^-T grad_xi phi
    gx = np.einsum("cqba,qib->cqia", Jinv, grad)    # (ncell, nq, nb, d)
    Ke = np.einsum("cq,cqia,cqja->cij", wdet, gx, gx)
    return Me, Ke


def assemble_deformed(mesh):
    """Assembled CSR M and K on all nodes (no elimination)."""
    Me, Ke = element_matrices_deformed(mesh)
    dofs = mesh.cell_dofs()
    nb = dofs.shape[1]
    rows = np.repeat(dofs, nb, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, nb)).reshape(-1)
    M = sp.coo_matrix((Me.reshape(-1), (rows, cols)), shape=(mesh.n, mesh.n)).tocsr()
    K = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(mesh.n, mesh.n)).tocsr()
    return M, K


def load_vector_deformed(mesh):
    """G_j = int S(x) phi_j dx over the curved cells (Gauss (k+1)^d); zero on the boundary."""
    xi, w, phi, _ = mesh.quadrature()
    det = np.linalg.det(jacobian(xi, mesh.eps))
    Sq = S_exact(phi_map(xi, mesh.eps))             # source profile at the physical points
    Ge = (Sq * det * w[None, :]) @ phi
    dofs = mesh.cell_dofs()
    G = np.bincount(dofs.reshape(-1), weights=Ge.reshape(-1), minlength=mesh.n)
    G[mesh.boundary_mask()] = 0.0
    return G


def initial_value_deformed(mesh, t=0.0):
    """Interpolant of u(., t) at the mapped nodes (zero on the boundary)."""
    y = u_exact(mesh.node_coords(), t)
    y[mesh.boundary_mask()] = 0.0
    return y


def l2_error_deformed(mesh, y, t, extra=3):
    """|| u_h - u(t) ||_{L2} over the curved cells, (k+1+extra)-point Gauss per cell."""
    xi, w, phi, _ = mesh.quadrature(mesh.p + extra)
    det = np.linalg.det(jacobian(xi, mesh.eps))
    uh = y[mesh.cell_dofs()] @ phi.T
    err = uh - u_exact(phi_map(xi, mesh.eps), t)
    return float(np.sqrt(np.sum(err ** 2 * det * w[None, :])))


class DeformedProblem:
    """Heat problem on DeformedMesh(d, N, k, eps), Radau IIA with Q stages, step tau.

    Same interface as oracle.irk.Problem (apply_M, apply_K, y0, stage_loads, assemble), so that
    oracle.irk.apply_calA and oracle.irk.step_direct take it unchanged."""

    def __init__(self, d, N, k, Q, tau, eps):
        self.mesh = DeformedMesh(d, N, k, eps)
        self.d, self.N, self.k, self.Q, self.tau, self.eps = d, N, k, Q, tau, eps
        self.A, self.b, self.c = radau_iia(Q)
        self.Ainv = np.linalg.inv(self.A)
        self.G = load_vector_deformed(self.mesh)
        self._Me = self._Ke = None

    def element_mats(self):
        if self._Me is None:
            self._Me, self._Ke = element_matrices_deformed(self.mesh)
        return self._Me, self._Ke

    def _apply(self, Ce, u):
        mesh = self.mesh
        bmask = mesh.boundary_mask()
        u = np.array(u, dtype=np.float64, copy=True)
        u[..., bmask] = 0.0
        dofs = mesh.cell_dofs()
        lead = u.shape[:-1]
        uflat = u.reshape(-1, mesh.n)
        v = np.zeros_like(uflat)
        for s in range(uflat.shape[0]):
            ve = np.einsum("cij,cj->ci", Ce, uflat[s][dofs])
            v[s] = np.bincount(dofs.reshape(-1), weights=ve.reshape(-1), minlength=mesh.n)
        v[:, bmask] = 0.0
        return v.reshape(lead + (mesh.n,))

    def apply_M(self, u):
        return self._apply(self.element_mats()[0], u)

    def apply_K(self, u):
        return self._apply(self.element_mats()[1], u)

    def assemble(self):
        return assemble_deformed(self.mesh)

    def y0(self):
        return initial_value_deformed(self.mesh, 0.0)

    def stage_loads(self, t_n):
        return np.stack([phi_time(self.d, t_n + ci * self.tau) * self.G for ci in self.c])

    def stage_rhs_kron(self, y_n, t_n):
        return self.stage_loads(t_n) - self.apply_K(y_n)[None, :]

    def stage_rhs_calA(self, y_n, t_n):
        return self.Ainv @ self.stage_rhs_kron(y_n, t_n)
