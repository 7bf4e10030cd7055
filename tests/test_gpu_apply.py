"""Parity of the matrix-free sum-factorised operator kernels with the oracle (FP64, <= 1e-12).

The oracle applies the dense (k+1)^d element matrices cell by cell (no sum
factorisation); the GPU applies the stage operator of Eq. (irk:A) and the
general (Cm (x) M + Ck (x) K) form with its tensor-product kernels.  Sizes
span several CTA tiles in x, y and z with ragged tails.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.irk import Problem, apply_calA
from synthetic import HEAT3D_K4_N32_Q3, uniform_vectors, zero_boundary
from tests.gpu_util import from_dev, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12

# (dim, cells, degree, stages): several CTA tiles in x (32 cells in 3D, 64 in 2D), y and z,
# ragged tails, odd cell counts (coarsest level solved by fast diagonalisation)
CASES = [(2, 70, 1, 2), (2, 37, 2, 3), (2, 20, 3, 2), (2, 66, 4, 3),
         (3, 66, 1, 2), (3, 36, 2, 3), (3, 12, 2, 2), (3, 34, 3, 3), (3, 40, 4, 2), (3, 5, 4, 5)]


def _inputs(Q, dim, n1, seed=0):
    return zero_boundary(uniform_vectors((Q, n1 ** dim), seed=seed), dim, n1)


@pytest.mark.parametrize("dim,N,k,Q", CASES)
@pytest.mark.parametrize("op_ff", [1, 0])
def test_calA_apply(dim, N, k, Q, op_ff):
    """Float-float (default) and native FP64 evaluation of the operator, both <= 1e-12."""
    tau = 1e-2
    prob = Problem(dim, N, k, Q, tau)
    with pkg.Solver(dim, N, k, Q, tau, op_ff=op_ff) as s:
        u = _inputs(Q, dim, k * N + 1)
        ud = to_dev(s, u)
        vd = torch.zeros_like(ud)
        s.apply(ud, vd)
        got = from_dev(vd, s.n)
    ref = apply_calA(prob, u)
    assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("dim,N,k", [(2, 9, 3), (3, 7, 2), (3, 33, 1)])
def test_general_operator(dim, N, k):
    """v = (Cm (x) M + Ck (x) K) u with full coupling matrices (e.g. the 2x2 block of Sec. 6)."""
    tau = 3e-3
    rng = np.random.default_rng(5)
    Cm = rng.standard_normal((2, 2))
    Ck = rng.standard_normal((2, 2))
    prob = Problem(dim, N, k, 2, tau)
    with pkg.Solver(dim, N, k, 2, tau) as s:
        u = _inputs(2, dim, k * N + 1, seed=3)
        ud = to_dev(s, u)
        vd = torch.zeros_like(ud)
        s.apply_op(ud, vd, Cm, Ck)
        got = from_dev(vd, s.n)
    ref = Cm @ prob.apply_M(u) + Ck @ prob.apply_K(u)
    assert rel_err(got, ref) <= TOL


def test_boundary_entries_untouched():
    dim, N, k, Q = 3, 6, 3, 2
    with pkg.Solver(dim, N, k, Q, 1e-2) as s:
        u = to_dev(s, _inputs(Q, dim, k * N + 1))
        v = torch.full_like(u, 0.0)
        s.apply(u, v)
        got = from_dev(v, s.n)
    bmask = zero_boundary(np.ones(s.n), dim, k * N + 1) == 0
    assert np.all(got[:, bmask] == 0.0)


@pytest.mark.slow
@pytest.mark.parametrize("op_ff", [1, 0])
def test_calA_apply_full_size(op_ff):
    """The bench workload (3D, k=4, 32^3 cells, Q=3), every output compared."""
    w = HEAT3D_K4_N32_Q3
    prob = Problem(w.dim, w.cells, w.degree, w.Q, w.tau)
    with pkg.Solver(w.dim, w.cells, w.degree, w.Q, w.tau, op_ff=op_ff) as s:
        u = _inputs(w.Q, w.dim, w.n1, seed=11)
        ud = to_dev(s, u)
        vd = torch.zeros_like(ud)
        s.apply(ud, vd)
        got = from_dev(vd, s.n)
    ref = apply_calA(prob, u)
    assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("op_ff", [1, 0])
def test_calA_apply_smooth_input(op_ff):
    """Smooth input (the initial interpolant per stage): the stiffness part cancels strongly."""
    from oracle.heat import initial_value
    from oracle.fem import Mesh
    dim, N, k, Q, tau = 3, 16, 3, 3, 1e-3
    prob = Problem(dim, N, k, Q, tau)
    y = initial_value(Mesh(dim, N, k))
    u = np.stack([y * (1.0 + 0.1 * i) for i in range(Q)])
    with pkg.Solver(dim, N, k, Q, tau, op_ff=op_ff) as s:
        ud = to_dev(s, u)
        vd = torch.zeros_like(ud)
        s.apply(ud, vd)
        got = from_dev(vd, s.n)
    assert rel_err(got, apply_calA(prob, u)) <= TOL
