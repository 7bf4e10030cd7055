"""The paper's own workload of Sec. 5 through the C ABI, and its outer iteration counts.

u = prod sin(2 pi x_a) (1 + sin pi t) e^{-t/2}, tau = 0.1, loads handed to irk_step as stage loads.
1. The step equals the oracle's exact IRK step on these loads (1e-9, as every step test).
2. Cross-check with Table tab:complex:vs (k = 1, GMRES residual reduced by 1e12, IRK column):
   the LU-based preconditioner of Eq. (irk:P) with (nearly) exact block solves — FP64 multigrid,
   Chebyshev degree 16 — needs about the GMRES iterations the paper reports (5.0, 7.0, 9.9, 11.9
   for Q = 2, 4, 6, 8); the paper's counts belong to its own GMG, so the bar is a band around them.
   One degree-5 V-cycle per block (FP32 up to Q = 5, FP64 above, the default) stays within +2 of
   the same column on 64^3 cells.
3. The directly diagonalised variant with one V-cycle on each coupled 2x2 block (the paper's
   IRK-GMG column) needs at most the paper's iterations.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle import paper_workload as pw
from oracle.irk import FastDiag, Problem, step_fastdiag
from tests.gpu_util import rel_err, to_dev

pytestmark = pytest.mark.gpu

PAPER_ITS = {2: 5.0, 4: 7.0, 6: 9.9, 8: 11.9}  # Table tab:complex:vs, IRK, k = 1, L = 8
PAPER_ITS_GMG2 = {2: 7.0, 4: 14.0, 6: 22.0, 8: 31.3}  # the same table, IRK-GMG (one V-cycle on each 2x2 block)


def _steps(d, N, k, Q, tau, nsteps, **opts):
    prob = Problem(d, N, k, Q, tau)
    G2 = pw.load_vector(prob.mesh)
    fd = FastDiag(prob)
    yref = pw.initial_value(prob.mesh)
    its = []
    with pkg.Solver(d, N, k, Q, tau, stream=torch.cuda.Stream(), **opts) as s:
        y = s.vector()
        y.copy_(torch.from_numpy(pw.initial_value(prob.mesh)))
        for n in range(nsteps):
            t = n * tau
            loads = pw.stage_loads(prob, G2, t)
            g = to_dev(s, loads)
            torch.cuda.synchronize()
            its.append(s.step(y, t, stage_load=g).iterations)
            yref = step_fastdiag(prob, yref, t, fd, stage_loads=loads)
        s.synchronize()
        got = y.cpu().numpy()
    return rel_err(got, yref), its


@pytest.mark.parametrize("d,N,k,Q", [(3, 16, 1, 4), (3, 8, 4, 3), (3, 12, 2, 2)])
def test_paper_workload_step_matches_oracle(d, N, k, Q):
    err, its = _steps(d, N, k, Q, 0.1, 2)
    assert err <= 1e-9, (err, its)


@pytest.mark.slow
@pytest.mark.parametrize("Q", [2, 4, 6, 8])
def test_lu_preconditioner_iteration_counts_match_the_paper(Q):
    err, its = _steps(3, 32, 1, Q, 0.1, 2, rtol=1e-12, mg_precision=64, cheb_degree=16, max_it=400)
    assert err <= 1e-9, (err, its)
    paper = PAPER_ITS[Q]
    assert paper - 3 <= np.mean(its) <= paper + 2, (Q, its, paper)


@pytest.mark.slow
@pytest.mark.parametrize("Q", [2, 4, 6, 8])
def test_degree5_vcycle_iteration_counts_match_the_paper(Q):
    """One V-cycle of Chebyshev degree 5 per block (the paper's solver setup, Sec. 5) on 64^3 cells,
    default options otherwise: FP32 V-cycle up to Q = 5, FP64 from Q = 6 (where the basis change S~
    of Eq. irk:P would magnify FP32 rounding).  The outer iterations stay within +2 of the paper's
    IRK column (and not far below it)."""
    err, its = _steps(3, 64, 1, Q, 0.1, 2, rtol=1e-12, cheb_degree=5, max_it=400)
    assert err <= 1e-9, (err, its)
    paper = PAPER_ITS[Q]
    assert paper - 3 <= np.mean(its) <= paper + 2, (Q, its, paper)


@pytest.mark.slow
@pytest.mark.parametrize("Q", [2, 4, 6, 8])
def test_coupled_gmg_iteration_counts_vs_the_paper(Q):
    """Directly diagonalised variant with one V-cycle per 2x2 block (Sec. 6): the summed GMRES
    iterations over the blocks stay at or below the paper's IRK-GMG column (+2)."""
    err, its = _steps(3, 32, 1, Q, 0.1, 2, rtol=1e-12, cheb_degree=5, max_it=600,
                      variant=pkg.IRK_VARIANT_DIAG, pair_precond=1)
    assert err <= 1e-9, (err, its)
    assert np.mean(its) <= PAPER_ITS_GMG2[Q] + 2, (Q, its, PAPER_ITS_GMG2[Q])
