"""One Radau IIA step of the semi-discrete heat equation, solved exactly (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sources in arXiv 2209.06700, Sec. 2: for M u' + K u = g(t), the stage
vectors k = (k_1..k_Q) solve the Kronecker system
    (I_Q (x) M + tau A_Q (x) K) k = gbar - (I_Q (x) K)(1_Q (x) y_n),
gbar_i = g(t_n + c_i tau), and y_{n+1} = y_n + tau sum_i b_i k_i (Sec. 1).
Multiplying by (A_Q^{-1} (x) I) gives Eq. (irk:A) with the operator
    calA = A_Q^{-1} (x) M + tau I_Q (x) K,
whose action ``apply_calA`` is the operator the GPU path applies matrix-free.

Reading of the right-hand side sign: the printed stage system carries
"+ K u_0"; with k_i = f(t, y) = M^{-1}(g - K y) (Sec. 1 and 2 together) the
consistent sign is minus.  Backward Euler (Q = 1) and the convergence
orders in the tests confirm it.  e_Q in the printed RHS is read as the
all-ones vector 1_Q.

Three independent routes, all exact up to rounding:
* ``step_direct``: assemble the full Kronecker matrix on interior DoFs and
  solve it with a sparse direct solver (small meshes).
* ``step_fastdiag``: on the uniform mesh with Gauss (k+1)^d, M and K are
  exactly Kronecker products of the 1D matrices; the generalised 1D
  eigenproblem K1 V = M1 V diag(mu) decouples the system into scalar modes
  y' + mu y = ghat(t), on which the Q-stage step is a Q x Q solve per mode
  (Lynch, Rice and Thomas' fast diagonalisation; any size).
* ``exact_semidiscrete``: the closed-form solution of the modal ODEs, used
  for the temporal order 2Q-1.

Pinned by tests/test_oracle_irk.py: Q=1 equals backward Euler; direct ==
fast diagonalisation; Kronecker structure of M and K; temporal order 2Q-1
against the exact semi-discrete solution; spatial order k+1.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Mesh, assemble, apply_cellwise, element_matrices, interior_restrict
from .heat import initial_value, load_vector, phi_time
from .tableau import radau_iia


class Problem:
    """Heat problem on Mesh(d, N, k), Radau IIA with Q stages, step tau."""

    def __init__(self, d, N, k, Q, tau):
        self.mesh = Mesh(d, N, k)
        self.d, self.N, self.k, self.Q, self.tau = d, N, k, Q, tau
        self.A, self.b, self.c = radau_iia(Q)
        self.Ainv = np.linalg.inv(self.A)
        self.G = load_vector(self.mesh)
        self._Me = self._Ke = None

    def element_mats(self):
        if self._Me is None:
            self._Me, self._Ke = element_matrices(self.d, self.k, self.mesh.h)
        return self._Me, self._Ke

    def apply_M(self, u):
        Me, _ = self.element_mats()
        return apply_cellwise(self.mesh, Me, u)

    def apply_K(self, u):
        _, Ke = self.element_mats()
        return apply_cellwise(self.mesh, Ke, u)

    def y0(self):
        return initial_value(self.mesh, 0.0)

    def stage_loads(self, t_n):
        """gbar: (Q, n) with gbar_i = phi(t_n + c_i tau) G."""
        return np.stack([phi_time(self.d, t_n + ci * self.tau) * self.G for ci in self.c])

    def stage_rhs_kron(self, y_n, t_n):
        """Right-hand side of the un-transformed stage system: gbar_i - K y_n."""
        Ky = self.apply_K(y_n)
        return self.stage_loads(t_n) - Ky[None, :]

    def stage_rhs_calA(self, y_n, t_n):
        """Right-hand side of Eq. (irk:A): (A^{-1} (x) I)(gbar - 1 (x) K y_n)."""
        return self.Ainv @ self.stage_rhs_kron(y_n, t_n)


def apply_calA(prob, u, C=None, beta=None):
    """v_i = sum_j C_ij M u_j + beta K u_i with C = A^{-1}, beta = tau by default (Eq. irk:A)."""
    C = prob.Ainv if C is None else np.asarray(C)
    beta = prob.tau if beta is None else beta
    Mu = prob.apply_M(u)
    Ku = prob.apply_K(u)
    return C @ Mu + beta * Ku


def step_direct(prob, y_n, t_n, return_stages=False, stage_loads=None):
    """Exact step by a sparse direct solve of the Kronecker stage system (interior DoFs).

    stage_loads: optional (Q, n) array g(t_n + c_i tau) replacing the built-in source."""
    mesh = prob.mesh
    M, K = prob.assemble() if hasattr(prob, "assemble") else assemble(mesh)
    MI, keep = interior_restrict(mesh, M)
    KI, _ = interior_restrict(mesh, K)
    Q, tau = prob.Q, prob.tau
    big = sp.kron(sp.identity(Q), MI) + tau * sp.kron(sp.csr_matrix(prob.A), KI)
    if stage_loads is None:
        rhs = prob.stage_rhs_kron(y_n, t_n)[:, keep].reshape(-1)
    else:
        rhs = (np.asarray(stage_loads) - prob.apply_K(y_n)[None, :])[:, keep].reshape(-1)
    kk = spla.spsolve(big.tocsc(), rhs).reshape(Q, -1)
    y1 = y_n.copy()
    y1[keep] = y_n[keep] + tau * (prob.b @ kk)
    if return_stages:
        full = np.zeros((Q, mesh.n))
        full[:, keep] = kk
        return y1, full
    return y1


class FastDiag:
    """Fast diagonalisation of M, K on the uniform mesh (exact Kronecker structure)."""

    def __init__(self, prob):
        self.prob = prob
        d, N, k = prob.d, prob.N, prob.k
        m1 = Mesh(1, N, k)
        M1, K1 = assemble(m1)
        M1I, _ = interior_restrict(m1, M1)
        K1I, _ = interior_restrict(m1, K1)
        self.M1 = M1I.toarray()
        self.K1 = K1I.toarray()
        mu, V = sla.eigh(self.K1, self.M1)
        self.mu1, self.V = mu, V
        self.ni = self.M1.shape[0]
        grids = np.meshgrid(*([mu] * d), indexing="ij")
        self.mu = sum(grids)  # axes in order (axis0, axis1, ...) = (x, y, z)
        mesh = prob.mesh
        self.keep = np.flatnonzero(~mesh.boundary_mask())

    def _to_grid(self, vec_interior):
        # interior vector, x fastest -> array indexed [x, y, z]
        shape = (self.ni,) * self.prob.d
        return vec_interior.reshape(shape[::-1]).transpose()

    def _from_grid(self, arr):
        return arr.transpose().reshape(-1)

    def _axes_apply(self, B, arr):
        for a in range(arr.ndim):
            arr = np.moveaxis(np.tensordot(B, arr, axes=([1], [a])), 0, a)
        return arr

    def to_modal_state(self, y_full):
        """yhat = W^T M y with W = V (x) ... (x) V."""
        B = self.V.T @ self.M1
        return self._axes_apply(B, self._to_grid(y_full[self.keep]))

    def to_modal_load(self, g_full):
        """ghat = W^T g."""
        return self._axes_apply(self.V.T, self._to_grid(g_full[self.keep]))

    def from_modal(self, yhat):
        out = np.zeros(self.prob.mesh.n)
        out[self.keep] = self._from_grid(self._axes_apply(self.V, yhat))
        return out


def step_fastdiag(prob, y_n, t_n, fd=None, stage_loads=None):
    """Exact IRK step per mode: (I + tau mu A) khat = ghat_i - mu yhat 1, ghat_i the modal stage loads
    (phi(t_n + c_i tau) Ghat for the built-in source, or the given (Q, n) stage_loads)."""
    fd = FastDiag(prob) if fd is None else fd
    Q, tau = prob.Q, prob.tau
    yhat = fd.to_modal_state(y_n).reshape(-1)
    mu = fd.mu.reshape(-1)
    if stage_loads is None:
        Ghat = fd.to_modal_load(prob.G).reshape(-1)
        phis = np.array([phi_time(prob.d, t_n + ci * tau) for ci in prob.c])
        ghat = phis[None, :] * Ghat[:, None]                             # (nmodes, Q)
    else:
        ghat = np.stack([fd.to_modal_load(g).reshape(-1) for g in np.asarray(stage_loads)], axis=1)
    rhs = ghat - (mu * yhat)[:, None]                                    # (nmodes, Q)
    mats = np.eye(Q)[None, :, :] + tau * mu[:, None, None] * prob.A[None, :, :]
    khat = np.linalg.solve(mats, rhs[:, :, None])[:, :, 0]
    y1hat = yhat + tau * khat @ prob.b
    return fd.from_modal(y1hat.reshape(fd.mu.shape))


def exact_semidiscrete(prob, y0, T, fd=None):
    """Closed-form solution of M y' + K y = phi(t) G at time T from y(0) = y0.

    Per mode: y' + mu y = Ghat phi(t), phi(t) = Re[(d pi^2 + i) e^{it}], so
    y(T) = e^{-mu T} y0 + Ghat Re[(d pi^2 + i)(e^{iT} - e^{-mu T}) / (mu + i)].
    """
    fd = FastDiag(prob) if fd is None else fd
    yhat = fd.to_modal_state(y0)
    Ghat = fd.to_modal_load(prob.G)
    mu = fd.mu
    a = prob.d * np.pi ** 2 + 1j
    forced = np.real(a * (np.exp(1j * T) - np.exp(-mu * T)) / (mu + 1j))
    return fd.from_modal(np.exp(-mu * T) * yhat + Ghat * forced)


def run_steps(prob, nsteps, stepper="fastdiag", y0=None):
    """Advance nsteps from y0 (default: interpolant at t=0); returns y at t = nsteps*tau."""
    y = prob.y0() if y0 is None else y0.copy()
    fd = FastDiag(prob) if stepper == "fastdiag" else None
    for n in range(nsteps):
        t = n * prob.tau
        y = step_fastdiag(prob, y, t, fd) if fd is not None else step_direct(prob, y, t)
    return y
