"""Degenerate cases of the step: a zero state with zero loads, one stage (backward Euler), the
smallest meshes with a single interior node, against the oracle's exact step."""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.irk import FastDiag, Problem, step_fastdiag
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu


def test_zero_state_and_zero_loads_stay_zero():
    """rhs = 0: FGMRES returns at once (no iteration) and y_{n+1} = y_n = 0."""
    with pkg.Solver(3, 4, 2, 2, 1e-2) as s:
        y = s.vector()
        loads = s.stage_vector()
        st = s.step(y, 0.0, stage_load=loads)
        s.synchronize()
        assert st.iterations == 0
        assert torch.count_nonzero(y).item() == 0


@pytest.mark.parametrize("dim,N,k,Q,tau", [(2, 8, 2, 1, 1e-2), (3, 4, 3, 1, 1e-3),   # backward Euler
                                           (2, 1, 2, 2, 1e-2), (3, 1, 2, 3, 1e-2),   # one interior node
                                           (2, 2, 1, 2, 1e-2)])                      # one interior node, k = 1
def test_degenerate_step_matches_oracle(dim, N, k, Q, tau):
    prob = Problem(dim, N, k, Q, tau)
    yref = step_fastdiag(prob, prob.y0(), 0.0, FastDiag(prob))
    with pkg.Solver(dim, N, k, Q, tau) as s:
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        s.step(y, 0.0)
        s.synchronize()
        got = y.cpu().numpy()
    assert rel_err(got, yref) <= 1e-9


@pytest.mark.parametrize("dim,N,k,Q,tau,variant", [(2, 8, 2, 9, 1e-2, 0), (3, 4, 2, 9, 1e-3, 0),
                                                   (2, 8, 2, 9, 1e-2, 1), (3, 6, 4, 7, 1e-3, 0)])
def test_largest_stage_counts_match_oracle(dim, N, k, Q, tau, variant):
    """Q up to the largest the library takes (9; the FP64 V-cycle the default picks from Q = 6 on),
    in the LU and the directly diagonalised variant."""
    prob = Problem(dim, N, k, Q, tau)
    yref = step_fastdiag(prob, prob.y0(), 0.0, FastDiag(prob))
    with pkg.Solver(dim, N, k, Q, tau, variant=variant) as s:
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        s.step(y, 0.0)
        s.synchronize()
        got = y.cpu().numpy()
    assert rel_err(got, yref) <= 1e-9
