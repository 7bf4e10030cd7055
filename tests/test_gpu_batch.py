"""irk_solve_batch: several independent problems stepped concurrently.

Each item must give the oracle's exact IRK step (1e-9 relative, as irk_step)
and the same bits as stepping its handle alone with irk_step (the kernels and
reductions are deterministic, so concurrency may change timing only).
"""
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.irk import FastDiag, Problem, step_fastdiag
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu

YTOL = 1e-9

CASES = [(3, 8, 2, 3, 1e-3), (2, 16, 3, 2, 1e-2), (3, 6, 4, 4, 1e-3), (3, 12, 1, 5, 5e-4),
         (2, 32, 2, 3, 1e-3)]


def _solvers(cases, own_streams=True, **opts):
    out = []
    for (d, N, k, Q, tau) in cases:
        st = torch.cuda.Stream() if own_streams else None
        out.append(pkg.Solver(d, N, k, Q, tau, stream=st, **opts))
    return out


def _initial(solvers):
    ys = []
    for s in solvers:
        y = s.vector()
        s.interpolate_initial(y, 0.0)
        s.synchronize()
        ys.append(y)
    return ys


@pytest.mark.parametrize("own_streams", [True, False])
def test_batch_matches_oracle_and_single_steps(own_streams):
    solvers = _solvers(CASES, own_streams)
    try:
        ys = _initial(solvers)
        single = [y.clone() for y in ys]
        refs = [Problem(*c).y0() for c in CASES]
        fds = [FastDiag(Problem(*c)) for c in CASES]
        for n in range(2):
            t_ns = [n * c[4] for c in CASES]
            status, per = pkg.solve_batch(solvers, ys, t_ns)
            assert status == 0 and per == [0] * len(CASES), (status, per)
            for s, y, t in zip(solvers, single, t_ns):
                s.step(y, t)
            for i, c in enumerate(CASES):
                refs[i] = step_fastdiag(Problem(*c), refs[i], t_ns[i], fds[i])
        torch.cuda.synchronize()
        for i, c in enumerate(CASES):
            got = ys[i].cpu().numpy()
            assert rel_err(got, refs[i]) <= YTOL, (c, rel_err(got, refs[i]))
            assert torch.equal(ys[i], single[i]), c
    finally:
        for s in solvers:
            s.close()


def test_batch_repeated_handle_runs_items_in_order():
    """The same handle twice: its two items run one after the other, each a full step of its own y."""
    c = CASES[0]
    s = pkg.Solver(*c, stream=torch.cuda.Stream())
    other = pkg.Solver(*CASES[1], stream=torch.cuda.Stream())
    try:
        ya, yb, yo = _initial([s, s, other])
        status, per = pkg.solve_batch([s, other, s], [ya, yo, yb], [0.0, 0.0, c[4]])
        assert status == 0 and per == [0, 0, 0]
        prob = Problem(*c)
        fd = FastDiag(prob)
        y1 = step_fastdiag(prob, prob.y0(), 0.0, fd)
        # yb started from y0 as well but was stepped from t = tau: a different (still exact) step
        y1b = step_fastdiag(prob, prob.y0(), c[4], fd)
        torch.cuda.synchronize()
        assert rel_err(ya.cpu().numpy(), y1) <= YTOL
        assert rel_err(yb.cpu().numpy(), y1b) <= YTOL
    finally:
        s.close()
        other.close()


def test_batch_reports_each_failure_and_leaves_failed_y_unchanged():
    ok = pkg.Solver(*CASES[0], stream=torch.cuda.Stream())
    bad = pkg.Solver(3, 8, 2, 3, 1e-2, stream=torch.cuda.Stream(), max_it=1)
    try:
        y_ok, y_bad = _initial([ok, bad])
        before = y_bad.clone()
        status, per = pkg.solve_batch([ok, bad], [y_ok, y_bad], [0.0, 0.0])
        assert per[0] == 0 and per[1] == pkg._capi.IRK_ENOTCONV
        assert status == pkg._capi.IRK_ENOTCONV
        torch.cuda.synchronize()
        assert torch.equal(y_bad, before)
        prob = Problem(*CASES[0])
        assert rel_err(y_ok.cpu().numpy(), step_fastdiag(prob, prob.y0(), 0.0, FastDiag(prob))) <= YTOL
    finally:
        ok.close()
        bad.close()


def test_batch_empty_and_invalid():
    lib = pkg.lib()
    assert lib.irk_solve_batch(None, None, None, 0, None) == 0
    assert lib.irk_solve_batch(None, None, None, 1, None) == pkg._capi.IRK_EINVAL
    assert lib.irk_solve_batch(None, None, None, -1, None) == pkg._capi.IRK_EINVAL
