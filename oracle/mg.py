"""Multigrid, Chebyshev and PRESB ingredients written from their definitions (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in arXiv 2209.06700:
* Sec. 5 (solver setup): each block (lambda_i M + tau K) of Eq. (irk:P) is
  approximated by one geometric-multigrid V-cycle; the smoother is a
  Chebyshev iteration around point-Jacobi; the paper's coarse solver (AMG)
  is replaced here by an exact dense solve.
* Sec. 6, Eq. (presb:p): the PRESB preconditioner of the 2x2 real block
  [[K', -M'], [M', K']] and its three-factor form.

Readings (the paper defers the multigrid details to its reference on
global-coarsening GMG):
* levels are the uniform meshes N, N/2, ... down to the first odd N or the
  smallest N with an interior node; the same degree k on every level; level
  operators are rediscretised (lambda M_l + tau K_l);
* prolongation is the Q_k embedding (coarse function evaluated at the fine
  nodes); restriction is its transpose;
* the Chebyshev iteration of degree m takes m steps of the three-term
  recurrence x_{j+1} = x_j + d_j,
      d_0 = r_0 / theta,  d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) r_j,
      r_j = D^{-1}(b - A x_j),  rho_0 = delta/theta,  rho_j = 1/(2 theta/delta - rho_{j-1}),
  over the eigenvalue interval [lo, hi] of D^{-1} A, theta = (hi+lo)/2,
  delta = (hi-lo)/2 (Saad's Chebyshev acceleration);
* one V(m, m)-cycle: pre-smooth from zero, residual, restrict, recurse,
  prolongate and add, post-smooth.

The coupled 2x2 V-cycle (``CoupledVCycle``, Sec. 6) is pinned by: with beta = 0 it is the
scalar V-cycle on each component; its nodal 2x2 Jacobi inverse inverts the nodal blocks; as a
stationary iteration it contracts the error of the coupled system.

Pinned by tests/test_oracle_mg.py: the Chebyshev error-propagation
polynomial equals T_m((theta - mu)/delta) / T_m(theta/delta) on every
eigenpair of D^{-1}A; the prolongation reproduces degree-k polynomials
exactly; <P^T r, v> = <r, P v>; the V-cycle is symmetric and its two-grid
error contraction is below one; the PRESB factors multiply to P and the
PRESB-preconditioned spectrum lies in [1/2, 1]; the sparse prolongation and level operator
(for meshes beyond the dense forms' reach) equal the dense definitions on small meshes.
The chosen Chebyshev interval and level count are heuristics:
parity unpinned beyond the algebraic checks above; only the converged step
result is pinned as a whole.
"""
import numpy as np
import scipy.linalg as sla

from .fem import Mesh, assemble, gll_nodes, interior_restrict, lagrange_values


def level_sizes(N, k):
    """Cells per direction on each level, fine to coarse."""
    nmin = 2 if k == 1 else 1
    sizes = [N]
    while sizes[-1] % 2 == 0 and sizes[-1] // 2 >= nmin:
        sizes.append(sizes[-1] // 2)
    return sizes


def prolongation(d, Nc, k):
    """Dense P (n_fine x n_coarse): coarse Q_k basis functions evaluated at fine nodes.

    Columns of coarse boundary nodes are zeroed (homogeneous Dirichlet).
    """
    mc, mf = Mesh(d, Nc, k), Mesh(d, 2 * Nc, k)
    xf = mf.node_coords()
    xi = gll_nodes(k)
    P = np.zeros((mf.n, mc.n))
    for f in range(mf.n):
        vals = [np.ones(1)]
        gidx = [np.zeros(1, dtype=np.int64)]
        for a in range(d):
            s = xf[f, a] * Nc
            c = min(int(np.floor(s)), Nc - 1)
            V, _ = lagrange_values(xi, np.array([s - c]))
            ga = (k * c + np.arange(k + 1)) * (mc.n1 ** a)
            vals = [np.outer(v, V[0]).reshape(-1) for v in vals]
            gidx = [(gi[:, None] + ga[None, :]).reshape(-1) for gi in gidx]
        P[f, gidx[0]] += vals[0]
    P[:, mc.boundary_mask()] = 0.0
    P[mf.boundary_mask(), :] = 0.0
    return P


def prolongation_1d(Nc, k):
    """Dense 1D Q_k embedding (kNf+1 x kNc+1), Nf = 2 Nc: coarse basis functions at the fine nodes
    of one grid line (no boundary elimination)."""
    mc, mf = Mesh(1, Nc, k), Mesh(1, 2 * Nc, k)
    xf = mf.node_coords_1d()
    xi = gll_nodes(k)
    P1 = np.zeros((mf.n1, mc.n1))
    for f in range(mf.n1):
        s = xf[f] * Nc
        c = min(int(np.floor(s)), Nc - 1)
        V, _ = lagrange_values(xi, np.array([s - c]))
        P1[f, k * c + np.arange(k + 1)] += V[0]
    return P1


def prolongation_sparse(d, Nc, k):
    """The prolongation of ``prolongation`` as a sparse matrix for larger meshes: on the uniform
    tensor-product mesh each Q_k basis function is a product of 1D ones, so P is the Kronecker
    product of the 1D embeddings (x fastest: P1 (x) .. (x) P1 with the z factor first), with the
    boundary rows and columns zeroed."""
    import scipy.sparse as sp
    P1 = sp.csr_matrix(prolongation_1d(Nc, k))
    P = P1
    for _ in range(d - 1):
        P = sp.kron(P1, P, format="csr")
    mc, mf = Mesh(d, Nc, k), Mesh(d, 2 * Nc, k)
    keep_f = sp.diags((~mf.boundary_mask()).astype(float))
    keep_c = sp.diags((~mc.boundary_mask()).astype(float))
    return (keep_f @ P @ keep_c).tocsr()


def level_operator_sparse(d, N, k, lam, tau):
    """lambda M + tau K as ``level_operator`` but sparse (CSR), boundary rows/columns zeroed."""
    import scipy.sparse as sp
    mesh = Mesh(d, N, k)
    M, K = assemble(mesh)
    b = mesh.boundary_mask()
    keep = sp.diags((~b).astype(float))
    return (keep @ (lam * M + tau * K) @ keep).tocsr(), b


def level_operator(d, N, k, lam, tau):
    """Assembled lambda M + tau K on interior DoFs embedded in full-length (dense for small N)."""
    mesh = Mesh(d, N, k)
    M, K = assemble(mesh)
    A = (lam * M + tau * K).toarray()
    b = mesh.boundary_mask()
    A[b, :] = 0.0
    A[:, b] = 0.0
    return A, b


def jacobi_diag(A, bmask):
    D = (A.diagonal() if hasattr(A, "tocsr") else np.diag(A)).copy()
    D[bmask] = 1.0
    return D


def chebyshev(A, D, b, x0, m, lo, hi, bmask):
    """Degree-m Chebyshev iteration around point-Jacobi (recurrence in the module header)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    x = x0.copy()
    r = (b - A @ x) / D
    r[bmask] = 0.0
    d = r / theta
    rho = delta / theta
    x = x + d
    for _ in range(1, m):
        rho_new = 1.0 / (2.0 * theta / delta - rho)
        r = (b - A @ x) / D
        r[bmask] = 0.0
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        x = x + d
        rho = rho_new
    return x


def max_eig_DinvA(A, D, bmask):
    """Largest eigenvalue of D^{-1} A on interior DoFs (dense symmetric form D^{-1/2} A D^{-1/2})."""
    keep = ~bmask
    Ai = A[np.ix_(keep, keep)]
    s = 1.0 / np.sqrt(D[keep])
    return float(sla.eigvalsh(s[:, None] * Ai * s[None, :])[-1])


class VCycle:
    """One V(m, m)-cycle for lambda M + tau K on the uniform hierarchy (FP64, dense, small N)."""

    def __init__(self, d, N, k, lam, tau, m, bounds=None, smoothing_range=10.0, safety=1.2):
        self.sizes = level_sizes(N, k)
        self.levels = []
        for li, Nl in enumerate(self.sizes):
            A, bm = level_operator(d, Nl, k, lam, tau)
            D = jacobi_diag(A, bm)
            if bounds is not None:
                lo, hi = bounds[li]
            else:
                hi = safety * max_eig_DinvA(A, D, bm)
                lo = hi / smoothing_range
            self.levels.append(dict(N=Nl, A=A, D=D, bm=bm, lo=lo, hi=hi))
        self.P = [prolongation(d, self.sizes[i + 1], k) for i in range(len(self.sizes) - 1)]
        c = self.levels[-1]
        keep = ~c["bm"]
        self.coarse_keep = keep
        self.coarse_inv = np.linalg.inv(c["A"][np.ix_(keep, keep)])
        self.m = m

    def coarse_solve(self, b):
        x = np.zeros_like(b)
        x[self.coarse_keep] = self.coarse_inv @ b[self.coarse_keep]
        return x

    def apply(self, b, level=0):
        if level == len(self.levels) - 1:
            return self.coarse_solve(b)
        L = self.levels[level]
        x = chebyshev(L["A"], L["D"], b, np.zeros_like(b), self.m, L["lo"], L["hi"], L["bm"])
        r = b - L["A"] @ x
        r[L["bm"]] = 0.0
        bc = self.P[level].T @ r
        ec = self.apply(bc, level + 1)
        x = x + self.P[level] @ ec
        x = chebyshev(L["A"], L["D"], b, x, self.m, L["lo"], L["hi"], L["bm"])
        return x


def coupled_level(d, N, k, alpha, beta, tau):
    """The 2x2 block of Sec. 6 (Eq. complex:twobytwo) on one level, for x = (x0, x1):
    [[alpha M + tau K, -beta M], [beta M, alpha M + tau K]], rediscretised, boundary rows and
    columns zeroed (dense, small N); with its nodal 2x2 Jacobi inverse (reading: the paper's
    point-Jacobi, applied to the coupled system, takes a node with its two components as the
    point)."""
    mesh = Mesh(d, N, k)
    M, K = assemble(mesh)
    M, K = M.toarray(), K.toarray()
    bm = mesh.boundary_mask()
    for X in (M, K):
        X[bm, :] = 0.0
        X[:, bm] = 0.0
    A = alpha * M + tau * K
    C = np.block([[A, -beta * M], [beta * M, A]])
    da = np.diag(A).copy()
    dm = beta * np.diag(M)
    da[bm] = 1.0
    dm[bm] = 0.0
    n = mesh.n

    def dinv(r):
        """z = blockdiag([[da_i, -dm_i], [dm_i, da_i]])^{-1} r, node by node."""
        r0, r1 = r[:n], r[n:]
        den = da * da + dm * dm
        z = np.concatenate([(da * r0 + dm * r1) / den, (da * r1 - dm * r0) / den])
        z[np.concatenate([bm, bm])] = 0.0
        return z

    return C, dinv, np.concatenate([bm, bm])


def chebyshev_op(A, dinv, b, x0, m, lo, hi, bmask):
    """The Chebyshev recurrence of ``chebyshev`` with a general inverse-diagonal map dinv."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    x = x0.copy()
    r = dinv(b - A @ x)
    r[bmask] = 0.0
    dd = r / theta
    rho = delta / theta
    x = x + dd
    for _ in range(1, m):
        rho_new = 1.0 / (2.0 * theta / delta - rho)
        r = dinv(b - A @ x)
        r[bmask] = 0.0
        dd = rho_new * rho * dd + (2.0 * rho_new / delta) * r
        x = x + dd
        rho = rho_new
    return x


class CoupledVCycle:
    """One V(m, m)-cycle on the coupled 2x2 system itself (Sec. 6: GMG applied directly to
    Eq. complex:twobytwo, the paper's IRK-GMG): per level the rediscretised coupled operator,
    Chebyshev around nodal 2x2 block Jacobi over the interval ``bounds[level]``, the Q_k
    prolongation per component, the coarsest coupled system solved exactly (FP64, dense)."""

    def __init__(self, d, N, k, alpha, beta, tau, m, bounds):
        self.sizes = level_sizes(N, k)
        self.levels = []
        for li, Nl in enumerate(self.sizes):
            C, dinv, bm = coupled_level(d, Nl, k, alpha, beta, tau)
            lo, hi = bounds[li] if li < len(bounds) else (1.0, 2.0)
            self.levels.append(dict(N=Nl, A=C, dinv=dinv, bm=bm, lo=lo, hi=hi))
        self.P = [prolongation(d, self.sizes[i + 1], k) for i in range(len(self.sizes) - 1)]
        c = self.levels[-1]
        keep = ~c["bm"]
        self.coarse_keep = keep
        self.coarse_inv = np.linalg.inv(c["A"][np.ix_(keep, keep)])
        self.m = m

    def _P2(self, level, e):
        P = self.P[level]
        nc = P.shape[1]
        return np.concatenate([P @ e[:nc], P @ e[nc:]])

    def _R2(self, level, r):
        P = self.P[level]
        nf = P.shape[0]
        return np.concatenate([P.T @ r[:nf], P.T @ r[nf:]])

    def apply(self, b, level=0):
        if level == len(self.levels) - 1:
            x = np.zeros_like(b)
            x[self.coarse_keep] = self.coarse_inv @ b[self.coarse_keep]
            return x
        L = self.levels[level]
        x = chebyshev_op(L["A"], L["dinv"], b, np.zeros_like(b), self.m, L["lo"], L["hi"], L["bm"])
        r = b - L["A"] @ x
        r[L["bm"]] = 0.0
        ec = self.apply(self._R2(level, r), level + 1)
        x = x + self._P2(level, ec)
        return chebyshev_op(L["A"], L["dinv"], b, x, self.m, L["lo"], L["hi"], L["bm"])


def presb_factors(Kp, Mp):
    """The three factors of Eq. (presb:p) and P itself (dense)."""
    n = Kp.shape[0]
    I = np.eye(n)
    Z0 = np.zeros((n, n))
    X = np.block([[I, -I], [Z0, I]])
    Y = np.block([[Kp + Mp, Z0], [Mp, Kp + Mp]])
    Z = np.block([[I, I], [Z0, I]])
    P = np.block([[Kp, -Mp], [Mp, Kp + 2 * Mp]])
    return X, Y, Z, P


def presb_apply(Hsolve, Mp_apply, f, g):
    """P^{-1} (f, g) by the factored form: two sequential solves with H = K' + M'."""
    a = f + g
    w1 = Hsolve(a)
    w2 = Hsolve(g - Mp_apply(w1))
    return w1 - w2, w2
