"""Parity of the 3D streaming level-operator kernels in every launch shape with the oracle.

The FP32 Chebyshev step and residual of the multigrid levels run in the z-streaming kernel on
levels of more than 8 cells per axis; its launch shape (cells per warp segment, cells per z chunk,
chunks of a tile as one thread-block cluster) is picked by the cost model or the autotuner.  Here
each shape is forced through irk_op_shape_force on 3D meshes of 16-24 cells per axis, the
smoother (Chebyshev degree 3, from a nonzero start and from zero) and the residual of every block
are compared element by element with the oracle's sparse level operator (Sec. 5 solver setup:
Chebyshev around point-Jacobi on lambda_i M + tau K), and irk_op_shape_last confirms the shape that
ran.  The transfers (Q_k embedding and its transpose, the x-row and axis-pass kernels) are
compared with the oracle's sparse prolongation on the same meshes.  At the bench's full sizes
(degree 4 on 32^3 cells, degree 3 on 64^3 cells) the residual and one Chebyshev step of the
finest level are compared at sampled nodes with the oracle's cell matrices around them.

Tolerances: FP32 arithmetic against the FP64 oracle, relative to the largest reference entry,
2e-5 for one operator application and 2e-4 for degree-3 smoothing (as in tests/test_gpu_mg.py).
The right-hand sides are scaled to the size of A x so that an operator error cannot hide under b.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.fem import Mesh, element_matrices
from oracle.mg import chebyshev, jacobi_diag, level_operator_sparse, level_sizes, prolongation_sparse
from oracle.tableau import lu_preconditioner_factors
from synthetic import uniform_vectors, zero_boundary
from tests.gpu_util import from_dev, rel_err, to_dev

pytestmark = pytest.mark.gpu

TAU = 1e-2
TOL_OP, TOL_SMOOTH = 2e-5, 2e-4


def _shapes(N):
    """Launch shapes (cxs, zc, cluster): every segment width, one and several chunks (ragged
    last chunk), clusters of 2..16 chunks."""
    out = [(32, 1, 0), (32, N, 0), (16, 3, 0), (16, 3, 1), (8, 5, 1), (8, 7, 0), (32, 2, 1),
           (16, (N + 1) // 2, 1), (32, 4, 1)]
    return [s for s in out if s[2] == 0 or 2 <= -(-N // s[1]) <= 16]


CASES = [(16, 4, 2), (24, 3, 3), (20, 2, 2)]


def _problem(N, k, Q, seed):
    lam = lu_preconditioner_factors(Q)["lam"]
    n1 = k * N + 1
    A = [level_operator_sparse(3, N, k, lam[i], TAU) for i in range(Q)]
    bm = A[0][1]
    x0 = zero_boundary(uniform_vectors((Q, n1 ** 3), seed=seed), 3, n1)
    ax = np.stack([A[i][0] @ x0[i] for i in range(Q)])
    b = zero_boundary(uniform_vectors((Q, n1 ** 3), seed=seed + 1), 3, n1)
    b *= np.abs(ax).max(axis=1, keepdims=True)
    return lam, A, bm, x0, b


@pytest.mark.parametrize("N,k,Q", CASES)
def test_streaming_smoother_and_residual_every_shape(N, k, Q):
    lam, A, bm, x0, b = _problem(N, k, Q, seed=31)
    n = (k * N + 1) ** 3
    res_ref = np.stack([b[i] - A[i][0] @ x0[i] for i in range(Q)])
    with pkg.Solver(3, N, k, Q, TAU, mg_precision=32, cheb_degree=3, autotune=0) as s:
        bounds = [s.cheb_interval(0, i) for i in range(Q)]
        sm_ref = {}
        for from_zero in (False, True):
            sm_ref[from_zero] = np.stack([
                chebyshev(A[i][0], jacobi_diag(A[i][0], bm), b[i], np.zeros(n) if from_zero else x0[i], 3,
                          bounds[i][0], bounds[i][1], bm) for i in range(Q)])
        bd = to_dev(s, b, torch.float32)
        try:
            for cxs, zc, cl in _shapes(N):
                pkg.op_shape_force(4, cxs, zc, cl)
                out = s.stage_vector(dtype=torch.float32)
                s.mg_residual(0, bd, to_dev(s, x0, torch.float32), out)
                assert rel_err(from_dev(out, n), res_ref) <= TOL_OP, (cxs, zc, cl)
                assert pkg.op_shape_last(4) == (cxs, zc, cl, -(-N // zc))
                for from_zero in (False, True):
                    xd = to_dev(s, np.zeros_like(x0) if from_zero else x0, torch.float32)
                    s.mg_smooth(0, bd, xd, int(from_zero))
                    assert rel_err(from_dev(xd, n), sm_ref[from_zero]) <= TOL_SMOOTH, (cxs, zc, cl, from_zero)
                    assert pkg.op_shape_last(4) == (cxs, zc, cl, -(-N // zc))
        finally:
            pkg.op_shape_force(4, 0)


@pytest.mark.parametrize("N,k,Q", CASES)
def test_second_level_streaming_shapes(N, k, Q):
    """Level 1 (N/2 = 8..12 cells: the narrow 16-cell segments) in its model shape and forced ones."""
    Nl = N // 2
    if Nl <= 8:
        pytest.skip("level 1 runs the cell kernel")
    lam, A, bm, x0, b = _problem(Nl, k, Q, seed=41)
    n = (k * Nl + 1) ** 3
    res_ref = np.stack([b[i] - A[i][0] @ x0[i] for i in range(Q)])
    with pkg.Solver(3, N, k, Q, TAU, mg_precision=32, autotune=0) as s:
        bd = to_dev(s, b, torch.float32, level=1)
        try:
            for shape in [None, (16, 1, 0), (16, 2, 1), (8, 3, 1), (32, Nl, 0)]:
                if shape:
                    pkg.op_shape_force(4, *shape)
                out = s.stage_vector(dtype=torch.float32, level=1)
                s.mg_residual(1, bd, to_dev(s, x0, torch.float32, level=1), out)
                assert rel_err(from_dev(out, n), res_ref) <= TOL_OP, shape
                if shape:
                    assert pkg.op_shape_last(4)[:3] == shape
        finally:
            pkg.op_shape_force(4, 0)


@pytest.mark.parametrize("N,k,Q", CASES)
def test_transfers_on_multi_tile_meshes(N, k, Q):
    sizes = level_sizes(N, k)
    with pkg.Solver(3, N, k, Q, TAU, mg_precision=32, autotune=0) as s:
        for lev in range(min(2, len(sizes) - 1)):
            Nf, Nc = sizes[lev], sizes[lev + 1]
            n1f, n1c = k * Nf + 1, k * Nc + 1
            P = prolongation_sparse(3, Nc, k)
            r = zero_boundary(uniform_vectors((Q, n1f ** 3), seed=50 + lev), 3, n1f)
            bc = s.stage_vector(dtype=torch.float32, level=lev + 1)
            s.mg_restrict(lev, to_dev(s, r, torch.float32, level=lev), bc)
            assert rel_err(from_dev(bc, n1c ** 3), (P.T @ r.T).T) <= TOL_OP
            e = zero_boundary(uniform_vectors((Q, n1c ** 3), seed=60 + lev), 3, n1c)
            x0 = zero_boundary(uniform_vectors((Q, n1f ** 3), seed=70 + lev), 3, n1f)
            xd = to_dev(s, x0, torch.float32, level=lev)
            s.mg_prolongate(lev, to_dev(s, e, torch.float32, level=lev + 1), xd)
            assert rel_err(from_dev(xd, n1f ** 3), x0 + (P @ e.T).T) <= TOL_OP


def _around(p, N, k):
    """Cells whose closure holds node p (3 grid indices) and the node's local index in each."""
    cand = [[c for c in (i // k - 1, i // k) if 0 <= c < N and k * c <= i <= k * (c + 1)] for i in p]
    return [((cx, cy, cz), (p[0] - k * cx) + (k + 1) * ((p[1] - k * cy) + (k + 1) * (p[2] - k * cz)))
            for cz in cand[2] for cy in cand[1] for cx in cand[0]]


@pytest.mark.slow
@pytest.mark.parametrize("N,k,Q", [(32, 4, 3), (64, 3, 3)])
def test_full_size_finest_level_at_sampled_nodes(N, k, Q):
    """The bench's finest levels in the launch shape the bench runs (the model's, which the
    autotuner confirms there): the residual and one Chebyshev step (x1 = x0 + D^-1 r / theta) at
    200 random interior nodes, against the oracle's cell matrices of the cells around each."""
    lam = lu_preconditioner_factors(Q)["lam"]
    n1 = k * N + 1
    n = n1 ** 3
    mesh = Mesh(3, N, k)
    Me, Ke = element_matrices(3, k, mesh.h)
    rng = np.random.default_rng(5)
    x0 = rng.uniform(-1.0, 1.0, (Q, n)).astype(np.float32).astype(np.float64)
    x0 = zero_boundary(x0, 3, n1)
    pts = rng.integers(1, n1 - 1, size=(200, 3))
    node = pts[:, 0] + n1 * (pts[:, 1] + n1 * pts[:, 2])
    # A x0 and diag(A) at the sampled nodes from the cells around them
    ax = np.zeros((Q, len(pts)))
    dg = np.zeros((Q, len(pts)))
    for j, p in enumerate(pts):
        for (cx, cy, cz), loc in _around(p, N, k):
            g = np.arange(k + 1)
            ids = ((k * cx + g)[None, None, :] + n1 * ((k * cy + g)[None, :, None] + n1 * (k * cz + g)[:, None, None]))
            xe = x0[:, ids.reshape(-1)]
            for i in range(Q):
                Ae = lam[i] * Me[loc] + TAU * Ke[loc]
                ax[i, j] += xe[i] @ Ae
                dg[i, j] += lam[i] * Me[loc, loc] + TAU * Ke[loc, loc]
    scale = np.abs(ax).max()
    b = zero_boundary(rng.uniform(-1.0, 1.0, (Q, n)) * scale, 3, n1).astype(np.float32).astype(np.float64)
    with pkg.Solver(3, N, k, Q, TAU, mg_precision=32, cheb_degree=1, autotune=0, restart=2) as s:
        bd, xd = to_dev(s, b, torch.float32), to_dev(s, x0, torch.float32)
        out = s.stage_vector(dtype=torch.float32)
        s.mg_residual(0, bd, xd, out)
        got_r = out[:, node].double().cpu().numpy()
        s.mg_smooth(0, bd, xd, 0)
        got_x = xd[:, node].double().cpu().numpy()
        theta = np.array([0.5 * sum(s.cheb_interval(0, i)) for i in range(Q)])
        shape = pkg.op_shape_last(4)
    ref_r = b[:, node] - ax
    ref_x = x0[:, node] + ref_r / dg / theta[:, None]
    assert rel_err(got_r, ref_r) <= TOL_OP
    assert rel_err(got_x, ref_x) <= TOL_OP
    assert shape[0] == 32 and shape[3] >= 1
