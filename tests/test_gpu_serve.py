"""Serving (irk_serve): continuous batching of single-step requests.

Each result must be the same alone and in the mix (the kernels, launch shapes and reductions of a
request do not depend on what else runs), agree with the oracle's exact step, and requests larger
than the memory budget are refused before any work.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.irk import Problem, step_fastdiag
from paper_2209_06700_gb300 import _capi

pytestmark = pytest.mark.gpu

# (dim, cells, degree, Q, tau, t0, arrival_s)
MIX = [(2, 16, 2, 2, 1e-2, 0.0, 0.000), (3, 8, 2, 3, 1e-3, 0.0, 0.001), (3, 8, 4, 4, 3e-3, 0.0, 0.002),
       (2, 32, 4, 3, 1e-4, 0.0, 0.003), (3, 16, 1, 2, 5e-3, 0.0, 0.004), (2, 8, 3, 4, 2e-3, 0.0, 0.005),
       (3, 6, 3, 3, 1e-3, 0.0, 0.006), (2, 64, 1, 2, 1e-2, 0.0, 0.007), (3, 12, 2, 2, 7e-4, 0.0, 0.008),
       (3, 16, 3, 3, 2e-4, 0.0, 0.009)]


def test_alone_equals_mix_and_oracle():
    st, res, ys = pkg.serve(MIX, max_active=6, realtime=False, outputs=True)
    assert st == 0, [r.status for r in res]
    assert all(r.status == 0 and r.iterations > 0 and r.latency_ms >= r.solve_ms > 0 for r in res)
    for i, req in enumerate(MIX):
        st1, res1, ys1 = pkg.serve([req], max_active=1, realtime=False, outputs=True)
        assert st1 == 0
        scale = np.abs(ys1[0]).max()
        assert np.abs(ys[i] - ys1[0]).max() <= 1e-12 * scale, i
        assert res1[0].iterations == res[i].iterations
    for i in (0, 2, 6):
        d, N, k, Q, tau, t0, _ = MIX[i]
        prob = Problem(d, N, k, Q, tau)
        ref = step_fastdiag(prob, prob.y0(), 0.0)
        assert np.abs(ys[i] - ref).max() <= 1e-9 * np.abs(ref).max(), i


# two shapes, several steps each: waiting requests of one shape run as a group with shared launches
SAME = [(3, 8, 2, 3, tau, t0, 0.0) for tau, t0 in ((1e-3, 0.0), (2e-3, 0.1), (5e-4, 0.2), (3e-3, 0.0))] + \
       [(2, 16, 3, 2, tau, 0.0, 0.0) for tau in (1e-2, 2e-3, 4e-4)]


def test_groups_share_launches_and_each_result_equals_alone():
    st, res, ys = pkg.serve(SAME, max_active=1, realtime=False, outputs=True)
    assert st == 0
    assert max(r.group_size for r in res) > 1, [r.group_size for r in res]
    for i, req in enumerate(SAME):
        st1, res1, ys1 = pkg.serve([req], max_active=1, realtime=False, outputs=True)
        assert st1 == 0 and res1[0].group_size == 1
        assert np.abs(ys[i] - ys1[0]).max() <= 1e-12 * np.abs(ys1[0]).max(), i
        assert res1[0].iterations == res[i].iterations
    # without groups and without handle reuse the results are the same
    st2, res2, ys2 = pkg.serve(SAME, max_active=2, realtime=False, outputs=True, max_group=1, reuse_handles=0)
    assert st2 == 0 and all(r.group_size == 1 and r.handle_reused == 0 for r in res2)
    for i in range(len(SAME)):
        assert np.abs(ys[i] - ys2[i]).max() <= 1e-12 * np.abs(ys2[i]).max(), i


def test_arrival_order_gives_the_same_results():
    st, res, ys = pkg.serve(SAME + MIX[:3], max_active=2, realtime=False, outputs=True)
    st2, res2, ys2 = pkg.serve(SAME + MIX[:3], max_active=2, realtime=False, outputs=True, smallest_first=0)
    assert st == 0 and st2 == 0
    for i in range(len(ys)):
        assert np.abs(ys[i] - ys2[i]).max() <= 1e-12 * np.abs(ys[i]).max(), i


def test_idle_handles_are_reused_for_later_requests():
    """One slot, groups of one: the second request of a shape takes the first one's handle (new
    tau set with irk_set_tau) and still matches the oracle."""
    reqs = [(3, 6, 3, 2, 1e-3, 0.0, 0.0), (3, 6, 3, 2, 4e-3, 0.0, 0.0), (3, 6, 3, 2, 2e-4, 0.0, 0.0)]
    st, res, ys = pkg.serve(reqs, max_active=1, realtime=False, outputs=True, max_group=1)
    assert st == 0
    assert res[0].handle_reused == 0 and res[1].handle_reused == 1 and res[2].handle_reused == 1
    for i, (d, N, k, Q, tau, t0, _) in enumerate(reqs):
        prob = Problem(d, N, k, Q, tau)
        ref = step_fastdiag(prob, prob.y0(), 0.0)
        assert np.abs(ys[i] - ref).max() <= 1e-9 * np.abs(ref).max(), i


def test_diagonalised_variant_is_served_request_by_request():
    """Groups need the LU variant: with the DIAG variant every request runs on its own handle and
    still matches the oracle."""
    reqs = [(3, 6, 2, 3, 1e-3, 0.0, 0.0), (3, 6, 2, 3, 2e-3, 0.0, 0.0), (2, 8, 3, 2, 5e-3, 0.0, 0.0)]
    st, res, ys = pkg.serve(reqs, max_active=2, realtime=False, outputs=True, variant=pkg.IRK_VARIANT_DIAG)
    assert st == 0 and all(r.group_size == 1 and r.handle_reused == 0 for r in res)
    for i, (d, N, k, Q, tau, t0, _) in enumerate(reqs):
        prob = Problem(d, N, k, Q, tau)
        ref = step_fastdiag(prob, prob.y0(), 0.0)
        assert np.abs(ys[i] - ref).max() <= 1e-9 * np.abs(ref).max(), i


def test_idle_handles_are_evicted_when_the_budget_needs_their_memory():
    """A budget that holds one handle at a time: alternating shapes evict the idle handle of the other
    shape (least recently used); every result still matches the oracle."""
    A, B = (3, 8, 2, 3, 1e-3, 0.0, 0.0), (3, 6, 3, 2, 2e-3, 0.0, 0.0)
    _, probe, _ = pkg.serve([A, B], max_active=1, realtime=False)
    ea, eb = probe[0].mem_bytes, probe[1].mem_bytes
    budget = 1.05 * max(ea, eb)
    if ea + eb <= budget:
        pytest.skip("the two requests fit together")
    reqs = [A, B, (3, 8, 2, 3, 4e-3, 0.0, 0.0), (3, 6, 3, 2, 5e-4, 0.0, 0.0)]
    # with room for both handles the last two requests reuse the first two's handles ...
    st, res, _ = pkg.serve(reqs, max_active=1, realtime=False, max_group=1, smallest_first=0)
    assert st == 0 and [r.handle_reused for r in res] == [0, 0, 1, 1]
    # ... with room for one, each request evicts the other shape's idle handle and creates its own
    st, res, ys = pkg.serve(reqs, max_active=1, realtime=False, outputs=True, mem_budget_bytes=budget,
                            max_group=1, smallest_first=0)
    assert st == 0 and [r.handle_reused for r in res] == [0, 0, 0, 0]
    for i, (d, N, k, Q, tau, t0, _) in enumerate(reqs):
        prob = Problem(d, N, k, Q, tau)
        ref = step_fastdiag(prob, prob.y0(), 0.0)
        assert np.abs(ys[i] - ref).max() <= 1e-9 * np.abs(ref).max(), i


def test_realtime_arrivals_and_latency_accounting():
    reqs = [(2, 16, 2, 2, 1e-2, 0.0, 0.01 * i) for i in range(6)]
    st, res, _ = pkg.serve(reqs, max_active=2, realtime=True)
    assert st == 0
    for r in res:
        assert r.queue_ms >= 0.0 and r.latency_ms >= r.queue_ms + r.setup_ms - 1e-6


def test_request_larger_than_budget_is_refused():
    st, res, _ = pkg.serve([(3, 16, 2, 2, 1e-3, 0.0, 0.0), (2, 8, 1, 2, 1e-3, 0.0, 0.0)], max_active=2,
                           realtime=False, mem_budget_bytes=8e6)
    assert res[0].status == _capi.IRK_EBUSY
    assert res[1].status == 0
    assert st == _capi.IRK_EBUSY


def test_nan_input_is_reported_and_leaves_y_unchanged():
    """Host-side fault injection: a NaN in y_n gives IRK_ENUMERIC and y is not modified."""
    with pkg.Solver(3, 6, 2, 3, 1e-3) as s:
        y = s.vector()
        torch.cuda.synchronize()
        s.interpolate_initial(y, 0.0)
        s.synchronize()
        idx = (2 * 6 + 1) ** 2 * 5 + (2 * 6 + 1) * 5 + 5
        y[idx] = float("nan")
        y0 = y.clone()
        with pytest.raises(pkg.IrkError) as ei:
            s.step(y, 0.0)
        assert ei.value.code == _capi.IRK_ENUMERIC
        assert torch.equal(torch.isnan(y), torch.isnan(y0))
        assert torch.equal(torch.nan_to_num(y), torch.nan_to_num(y0))
