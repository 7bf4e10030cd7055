"""The operator autotuner: shapes are timed at create, recorded, and leave results exact.

The tuner times candidate launch shapes (warp-segment width, z chunk, thread-block cluster) of
each 3D operator kernel on the handle's own buffers and keeps the fastest, process-wide.  Every
shape computes the same operator, so the step still matches the oracle's exact IRK step.
"""
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.irk import FastDiag, Problem, step_fastdiag
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu


def test_autotune_records_shapes_and_step_stays_exact():
    d, N, k, Q, tau = 3, 32, 2, 3, 1e-3  # 65^3 nodes x 3 stages: above the tuning threshold
    prob = Problem(d, N, k, Q, tau)
    with pkg.Solver(d, N, k, Q, tau, stream=torch.cuda.Stream(), autotune=1) as s:
        report = pkg.autotune_report()
        assert f"op3d<float> k={k} cheb N={N} stages={Q}" in report, report
        assert f"op3d<double> k={k} dual N={N} stages={Q}" in report, report   # native FP64 outer (default)
        for line in report.splitlines():
            assert " zc=" in line and " cluster=" in line
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        s.step(y, 0.0)
        s.synchronize()
        ref = step_fastdiag(prob, prob.y0(), 0.0, FastDiag(prob))
        assert rel_err(y.cpu().numpy(), ref) <= 1e-9


def test_autotune_off_uses_the_model_and_matches():
    d, N, k, Q, tau = 3, 12, 3, 2, 1e-3
    prob = Problem(d, N, k, Q, tau)
    with pkg.Solver(d, N, k, Q, tau, autotune=0) as s:
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        s.step(y, 0.0)
        s.synchronize()
        ref = step_fastdiag(prob, prob.y0(), 0.0, FastDiag(prob))
        assert rel_err(y.cpu().numpy(), ref) <= 1e-9
