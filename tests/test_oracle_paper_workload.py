"""Oracle pins for the paper's manufactured problem of Sec. 5 (CPU only).

u = prod sin(2 pi x_a) (1 + sin pi t) e^{-t/2}: the oracle's discretisation of this
problem converges at the spatial order k+1 to the analytic solution (which pins the
load vector G2, the time factor psi = theta' + 4 d pi^2 theta and the interpolant),
and its fast-diagonalised step with these stage loads equals the sparse direct
Kronecker solve.
"""
import numpy as np
import pytest

from oracle import paper_workload as pw
from oracle.irk import FastDiag, Problem, step_direct, step_fastdiag


def _run(prob, nsteps):
    G2 = pw.load_vector(prob.mesh)
    fd = FastDiag(prob)
    y = pw.initial_value(prob.mesh)
    for n in range(nsteps):
        t = n * prob.tau
        y = step_fastdiag(prob, y, t, fd, stage_loads=pw.stage_loads(prob, G2, t))
    return y


@pytest.mark.parametrize("k", [1, 2])
def test_spatial_order_on_the_paper_solution(k):
    errs = []
    for N in (8, 16, 32):
        prob = Problem(2, N, k, 5, 0.025)
        y = _run(prob, 4)
        errs.append(pw.l2_error(prob.mesh, y, 4 * prob.tau))
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - (k + 1)) < 0.2, (errs, rate)


@pytest.mark.parametrize("d,N,k,Q,tau", [(2, 4, 2, 3, 0.1), (3, 2, 2, 2, 0.1), (2, 3, 1, 4, 0.1)])
def test_fastdiag_equals_direct_with_the_paper_loads(d, N, k, Q, tau):
    prob = Problem(d, N, k, Q, tau)
    G2 = pw.load_vector(prob.mesh)
    y = pw.initial_value(prob.mesh)
    loads = pw.stage_loads(prob, G2, 0.3)
    a = step_fastdiag(prob, y, 0.3, stage_loads=loads)
    b = step_direct(prob, y, 0.3, stage_loads=loads)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_theta_prime_is_the_derivative():
    t = np.linspace(0.0, 2.0, 11)
    h = 1e-6
    fd = (pw.theta(t + h) - pw.theta(t - h)) / (2 * h)
    assert np.abs(fd - pw.theta_prime(t)).max() < 1e-8
