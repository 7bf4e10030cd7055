"""Parity of the curved-mesh path (the stage operator with mapping data at every Gauss point,
Sec. 3.4) with the oracle's dense per-cell quadrature on the same curved mesh.

Bars: operator applies 1e-12 relative; the initial interpolant and the stage right-hand side 1e-12;
the whole step 1e-9 relative in y_{n+1} against the oracle's sparse direct Kronecker solve; one
launch over all stages equals the per-stage launches bit for bit.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.deformed import DeformedProblem
from oracle.irk import apply_calA, step_direct
from synthetic import uniform_vectors, zero_boundary
from tests.gpu_util import from_dev, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12
YTOL = 1e-9

# (dim, cells, degree, stages, eps): several cells per axis, every degree, odd counts
CASES = [(2, 7, 1, 2, 0.1), (2, 6, 2, 3, 0.1), (2, 5, 4, 2, 0.1), (3, 5, 1, 2, 0.05), (3, 4, 2, 3, 0.05),
         (3, 3, 3, 2, 0.05), (3, 3, 4, 3, 0.05)]


def _inputs(Q, dim, n1, seed=0):
    return zero_boundary(uniform_vectors((Q, n1 ** dim), seed=seed), dim, n1)


@pytest.mark.parametrize("dim,N,k,Q,eps", CASES)
@pytest.mark.parametrize("op_ff", [1, 0])
def test_general_operator(dim, N, k, Q, eps, op_ff):
    """Float-float (default) and native FP64 arithmetic inside the curved-mesh operator."""
    rng = np.random.default_rng(7)
    Cm = rng.standard_normal((Q, Q))
    Ck = rng.standard_normal((Q, Q))
    prob = DeformedProblem(dim, N, k, Q, 1e-2, eps)
    with pkg.Solver(dim, N, k, Q, 1e-2, deform=eps, op_ff=op_ff) as s:
        u = _inputs(Q, dim, k * N + 1, seed=2)
        ud = to_dev(s, u)
        vd = torch.zeros_like(ud)
        s.apply_op(ud, vd, Cm, Ck)
        got = from_dev(vd, s.n)
    assert rel_err(got, Cm @ prob.apply_M(u) + Ck @ prob.apply_K(u)) <= TOL


@pytest.mark.parametrize("dim,N,k,Q,eps", CASES[1::2])
def test_calA_apply(dim, N, k, Q, eps):
    tau = 3e-3
    prob = DeformedProblem(dim, N, k, Q, tau, eps)
    with pkg.Solver(dim, N, k, Q, tau, deform=eps) as s:
        u = _inputs(Q, dim, k * N + 1, seed=4)
        ud = to_dev(s, u)
        vd = torch.zeros_like(ud)
        s.apply(ud, vd)
        got = from_dev(vd, s.n)
    assert rel_err(got, apply_calA(prob, u)) <= TOL


@pytest.mark.parametrize("op_ff", [1, 0])
def test_batched_launch_equals_per_stage_launches(op_ff):
    dim, N, k, Q, eps = 3, 5, 3, 3, 0.05
    Cm = np.diag([1.0, 2.0, 3.0])
    Ck = np.diag([0.5, 0.25, 0.125])
    with pkg.Solver(dim, N, k, Q, 1e-2, deform=eps, op_ff=op_ff) as s:
        ud = to_dev(s, _inputs(Q, dim, k * N + 1, seed=9))
        vb = torch.zeros_like(ud)
        s.apply_op(ud, vb, Cm, Ck)
        vs = torch.zeros_like(ud)
        for i in range(Q):
            s.apply_op(ud[i:i + 1], vs[i:i + 1], Cm[i:i + 1, i:i + 1], Ck[i:i + 1, i:i + 1])
        torch.cuda.synchronize()
        assert torch.equal(vb, vs)


@pytest.mark.parametrize("dim,N,k,Q", [(2, 8, 2, 3), (3, 4, 3, 2)])
@pytest.mark.parametrize("op_ff", [1, 0])
def test_initial_value_and_stage_rhs(dim, N, k, Q, op_ff):
    """On the smooth initial value the stiffness part of K y_n cancels strongly; the library
    evaluates K y_n in native FP64 whatever the operator's arithmetic, so both settings meet the
    1e-12 operator bar."""
    eps, tau = (0.1 if dim == 2 else 0.05), 1e-2
    prob = DeformedProblem(dim, N, k, Q, tau, eps)
    with pkg.Solver(dim, N, k, Q, tau, deform=eps, op_ff=op_ff) as s:
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        y0 = y.cpu().numpy()
        rhs = s.stage_vector()
        s.stage_rhs(y, 0.3, rhs)
        got = from_dev(rhs, s.n)
    assert rel_err(y0, prob.y0()) <= TOL
    assert rel_err(got, prob.stage_rhs_calA(prob.y0(), 0.3)) <= TOL


@pytest.mark.parametrize("dim,N,k,Q,tau,variant,op_ff", [(2, 8, 2, 3, 1e-2, 0, 1), (2, 6, 4, 2, 1e-2, 0, 1),
                                                         (3, 4, 2, 3, 1e-3, 0, 1), (3, 4, 3, 3, 1e-3, 0, 1),
                                                         (3, 4, 2, 3, 1e-3, 1, 1), (3, 4, 3, 3, 1e-3, 0, 0)])
def test_step(dim, N, k, Q, tau, variant, op_ff):
    eps = 0.1 if dim == 2 else 0.05
    prob = DeformedProblem(dim, N, k, Q, tau, eps)
    yref = prob.y0()
    with pkg.Solver(dim, N, k, Q, tau, deform=eps, variant=variant, op_ff=op_ff) as s:
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        its = []
        for n in range(2):
            its.append(s.step(y, n * tau).iterations)
            yref = step_direct(prob, yref, n * tau)
        s.synchronize()
        got = y.cpu().numpy()
    assert rel_err(got, yref) <= YTOL, its
    assert max(its) < 60, its


def test_invalid_amplitude_is_refused():
    with pytest.raises(pkg.IrkError):
        pkg.Solver(3, 4, 2, 2, 1e-2, deform=0.2)   # eps d pi >= 1: the map folds


@pytest.mark.slow
@pytest.mark.parametrize("op_ff", [1, 0])
def test_full_size_sampled_nodes(op_ff):
    """The bench's curved workload (3D, degree 4, 32^3 cells, Q = 3, eps = 0.05): M u and K u of
    every stage at 150 random interior nodes against the oracle's dense matrices of the cells
    around them (the full operator is out of reach of the dense oracle at this size)."""
    from oracle.deformed import DeformedMesh, element_matrices_deformed
    from synthetic import HEAT3D_K4_N32_Q3 as w
    eps = 0.05
    mesh = DeformedMesh(w.dim, w.cells, w.degree, eps)
    n1, n, Q, k, N = w.n1, w.n1 ** 3, w.Q, w.degree, w.cells
    u = _inputs(Q, 3, n1, seed=13)
    with pkg.Solver(3, N, k, Q, w.tau, deform=eps, op_ff=op_ff) as s:
        ud = to_dev(s, u)
        vm, vk = torch.zeros_like(ud), torch.zeros_like(ud)
        s.apply_op(ud, vm, np.eye(Q), np.zeros((Q, Q)))
        s.apply_op(ud, vk, np.zeros((Q, Q)), np.eye(Q))
        gm, gk = from_dev(vm, n), from_dev(vk, n)
    rng = np.random.default_rng(17)
    pts = rng.integers(1, n1 - 1, size=(150, 3))
    around = []
    for p in pts:   # the cells whose closure holds the node, and the node's local index in each
        cand = [[c for c in (i // k - 1, i // k) if 0 <= c < N and k * c <= i <= k * (c + 1)] for i in p]
        around.append([(cx + N * (cy + N * cz), (p[0] - k * cx) + (k + 1) * ((p[1] - k * cy) + (k + 1) * (p[2] - k * cz)))
                       for cz in cand[2] for cy in cand[1] for cx in cand[0]])
    cells = np.unique([c for a in around for c, _ in a])
    Me, Ke = element_matrices_deformed(mesh, cells=cells)
    slot = {c: i for i, c in enumerate(cells)}
    dofs = mesh.cell_dofs()
    node = pts[:, 0] + n1 * (pts[:, 1] + n1 * pts[:, 2])
    refm, refk = np.zeros((Q, len(pts))), np.zeros((Q, len(pts)))
    for j, a in enumerate(around):
        for c, loc in a:
            ue = u[:, dofs[c]]
            refm[:, j] += ue @ Me[slot[c], loc]
            refk[:, j] += ue @ Ke[slot[c], loc]
    assert rel_err(gm[:, node], refm) <= TOL
    assert rel_err(gk[:, node], refk) <= TOL
