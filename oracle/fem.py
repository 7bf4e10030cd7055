"""Continuous Q_k Lagrange finite elements on the uniform mesh of [0,1]^d (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in arXiv 2209.06700, Sec. 5 (setup of the numerical experiments):
the cube is refined uniformly into N cells per direction; continuous
Lagrange elements are tensor products of 1D elements of degree k; cell
integrals use the Gauss-Legendre rule with (k+1)^d points.  Sec. 2 gives the
semi-discrete system M u' + K u = g with mass matrix M and stiffness matrix K.

Readings (the paper is silent): the 1D element's nodes are the
Gauss-Lobatto-Legendre points; homogeneous Dirichlet conditions are imposed
by eliminating the boundary nodes (the full-length vectors keep a zero
there).  Global numbering is lexicographic over the (kN+1)^d node grid with
x fastest; a cell's local numbering is lexicographic with x fastest.

Everything is computed by direct quadrature from the definitions, with no
sum factorisation: the d-dimensional element matrices are built from basis
values at all (k+1)^d quadrature points, and the global operators are either
assembled to CSR (``assemble``) or applied cell by cell with the dense
element matrix (``apply_cellwise``).

Pinned by tests/test_oracle_fem.py: GLL nodes against closed forms;
symmetry and definiteness of M and K; sum(M) = 1 and K 1 = 0 before
elimination; polynomial exactness (mass of x^a y^b, energy of a quadratic);
CSR apply == cell-wise apply; spatial convergence order k+1 of the heat
solution (test_oracle_irk.py).
"""
import numpy as np
import scipy.sparse as sp


def gll_nodes(k):
    """Gauss-Lobatto-Legendre points of degree k on [0, 1] (k + 1 points)."""
    if k < 1:
        raise ValueError("degree k >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(k).deriv().roots()
    s = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (s + 1.0)


def gauss_rule(npts):
    """Gauss-Legendre points and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[q, i] = l_i(x_q) and D[q, i] = l_i'(x_q) for the Lagrange basis on ``nodes``."""
    x = np.asarray(x, dtype=np.float64)
    p = len(nodes)
    V = np.ones((len(x), p))
    D = np.zeros((len(x), p))
    for i in range(p):
        for m in range(p):
            if m == i:
                continue
            V[:, i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
        for m in range(p):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for l in range(p):
                if l == i or l == m:
                    continue
                term *= (x - nodes[l]) / (nodes[i] - nodes[l])
            D[:, i] += term
    return V, D


def element_matrices(d, k, h):
    """Dense element mass and stiffness matrices of one cube cell of side h.

    Direct Gauss quadrature with (k+1)^d points over the tensor-product basis.
    Returns (Me, Ke), each (k+1)^d x (k+1)^d.
    """
    p = k + 1
    xi = gll_nodes(k)
    xq, wq = gauss_rule(p)
    V, D = lagrange_values(xi, xq)
    nb = p ** d
    nq = p ** d
    # multi-indices, x fastest
    bidx = np.array(np.unravel_index(np.arange(nb), (p,) * d, order="F")).T  # (nb, d)
    qidx = np.array(np.unravel_index(np.arange(nq), (p,) * d, order="F")).T  # (nq, d)
    phi = np.ones((nq, nb))
    grad = np.ones((nq, nb, d))
    w = np.ones(nq)
    for a in range(d):
        Va = V[qidx[:, a]][:, bidx[:, a]]
        Da = D[qidx[:, a]][:, bidx[:, a]]
        phi *= Va
        w *= wq[qidx[:, a]]
        for g in range(d):
            grad[:, :, g] *= Da if g == a else Va
    # physical cell [0,h]^d: dx = h^d dxi, grad = grad_xi / h
    Me = (h ** d) * np.einsum("q,qi,qj->ij", w, phi, phi)
    Ke = (h ** (d - 2)) * np.einsum("q,qig,qjg->ij", w, grad, grad)
    return Me, Ke


class Mesh:
    """Uniform mesh of [0,1]^d with N cells per direction and Q_k nodes."""

    def __init__(self, d, N, k):
        if d not in (1, 2, 3):
            raise ValueError("d in {1, 2, 3}")
        self.d, self.N, self.k = d, N, k
        self.p = k + 1
        self.n1 = k * N + 1
        self.n = self.n1 ** d
        self.h = 1.0 / N

    def node_coords_1d(self):
        """Coordinate of every node of one grid line."""
        xi = gll_nodes(self.k)
        x = np.empty(self.n1)
        for c in range(self.N):
            for r in range(self.k + 1):
                x[c * self.k + r] = (c + xi[r]) * self.h
        return x

    def node_coords(self):
        """(n, d) array of node coordinates, x fastest."""
        x1 = self.node_coords_1d()
        # lexicographic with x fastest: index = x + n1*(y + n1*z)
        return np.stack([self._axis_coord(x1, a) for a in range(self.d)], axis=1)

    def _axis_coord(self, x1, axis):
        idx = np.arange(self.n)
        ia = (idx // (self.n1 ** axis)) % self.n1
        return x1[ia]

    def boundary_mask(self):
        idx = np.arange(self.n)
        mask = np.zeros(self.n, dtype=bool)
        for a in range(self.d):
            ia = (idx // (self.n1 ** a)) % self.n1
            mask |= (ia == 0) | (ia == self.n1 - 1)
        return mask

    def cell_dofs(self):
        """(ncells, p^d) global node index of every cell's local node (both x fastest)."""
        N, k, p, n1, d = self.N, self.k, self.p, self.n1, self.d
        cells = np.array(np.unravel_index(np.arange(N ** d), (N,) * d, order="F")).T
        loc = np.array(np.unravel_index(np.arange(p ** d), (p,) * d, order="F")).T
        out = np.zeros((N ** d, p ** d), dtype=np.int64)
        for a in range(d):
            out += (k * cells[:, a][:, None] + loc[:, a][None, :]) * (n1 ** a)
        return out


def assemble(mesh):
    """Assembled CSR mass and stiffness matrices on all nodes (no elimination)."""
    Me, Ke = element_matrices(mesh.d, mesh.k, mesh.h)
    dofs = mesh.cell_dofs()
    nb = dofs.shape[1]
    rows = np.repeat(dofs, nb, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, nb)).reshape(-1)
    ncell = dofs.shape[0]
    M = sp.coo_matrix((np.tile(Me.reshape(-1), ncell), (rows, cols)), shape=(mesh.n, mesh.n)).tocsr()
    K = sp.coo_matrix((np.tile(Ke.reshape(-1), ncell), (rows, cols)), shape=(mesh.n, mesh.n)).tocsr()
    return M, K


def interior_restrict(mesh, A):
    """Dirichlet elimination: keep interior rows/columns of an assembled matrix."""
    keep = np.flatnonzero(~mesh.boundary_mask())
    return A[keep][:, keep].tocsr(), keep


def apply_cellwise(mesh, Ce, u):
    """v = sum over cells of (gather, dense element matrix, scatter-add); boundary rows zeroed.

    ``u`` has shape (..., n); the boundary entries of ``u`` are treated as zero
    (Dirichlet elimination), and the returned ``v`` is zero on the boundary.
    """
    bmask = mesh.boundary_mask()
    u = np.array(u, dtype=np.float64, copy=True)
    u[..., bmask] = 0.0
    dofs = mesh.cell_dofs()
    lead = u.shape[:-1]
    uflat = u.reshape(-1, mesh.n)
    v = np.zeros_like(uflat)
    for s in range(uflat.shape[0]):
        ue = uflat[s][dofs]                # (ncell, nb)
        ve = ue @ Ce.T                     # (ncell, nb)
        v[s] = np.bincount(dofs.reshape(-1), weights=ve.reshape(-1), minlength=mesh.n)
    v[:, bmask] = 0.0
    return v.reshape(lead + (mesh.n,))
