"""Groups of requests in one handle (irk_create_group / irk_step_group): shared launches.

Several heat problems of the same shape, each with its own step tau and start time, share every
stage-operator and V-cycle launch while each keeps its own FGMRES.  Each request's y_{n+1} must
equal the result of a one-request handle (1e-12 relative; the launches take one request's launch
shape, so the per-stage arithmetic is the same) and the oracle's exact IRK step (1e-9); the
operator launches per step are those of the slowest request alone, not R times as many.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.heat import initial_value
from oracle.irk import Problem, step_fastdiag
from paper_2209_06700_gb300 import _capi

pytestmark = pytest.mark.gpu

YTOL = 1e-9


def _alone(dim, N, k, Q, tau, t0, y0, stream):
    with pkg.Solver(dim, N, k, Q, tau, stream=stream) as s:
        y = torch.from_numpy(y0).cuda()
        st = s.step(y, t0)
        s.synchronize()
        return y.cpu().numpy(), st.iterations


def _launches(s, cat):
    lib = _capi.lib()
    ms, n, nt = _capi.ctypes.c_double(), _capi.ctypes.c_longlong(), _capi.ctypes.c_longlong()
    lib.irk_profile_read(s.h, _capi.PROF_CATEGORIES.index(cat), _capi.ctypes.byref(ms), _capi.ctypes.byref(n),
                         _capi.ctypes.byref(nt))
    return n.value


@pytest.mark.parametrize("dim,N,k,Q,taus", [(3, 8, 2, 3, [1e-3, 4e-3, 2.5e-4]),
                                            (2, 16, 3, 2, [1e-2, 3e-3, 1e-4, 5e-3]),
                                            (3, 16, 4, 2, [1e-3] * 3 + [2e-3] * 3 + [5e-4, 8e-3])])
def test_group_equals_requests_alone_and_the_oracle(dim, N, k, Q, taus):
    R = len(taus)
    t0s = [0.1 * r for r in range(R)]
    stream = torch.cuda.Stream()
    probs = [Problem(dim, N, k, Q, tau) for tau in taus]
    y0s = [initial_value(p.mesh, t0s[r]) for r, p in enumerate(probs)]
    with pkg.Group(dim, N, k, Q, taus, stream=stream) as g:
        ys = [torch.from_numpy(y).cuda() for y in y0s]
        _capi.lib().irk_profile(g.h, 0)
        per, stats = g.step_group(ys, t0s)
        g.synchronize()
        assert per == [0] * R
        got = [y.cpu().numpy() for y in ys]
        its = [st.iterations for st in stats]
        op_launches = _launches(g, "apply64")
    for r in range(R):
        alone, its_alone = _alone(dim, N, k, Q, taus[r], t0s[r], y0s[r], stream)
        scale = np.abs(alone).max()
        assert np.abs(got[r] - alone).max() <= 1e-12 * scale, r
        assert its[r] == its_alone, (r, its, its_alone)
        ref = step_fastdiag(probs[r], y0s[r], t0s[r])
        assert np.abs(got[r] - ref).max() <= YTOL * np.abs(ref).max(), r
    # one stage-operator launch per FGMRES iteration of the slowest request, for all R requests
    assert op_launches == max(its), (op_launches, its)


def test_group_reuse_with_new_steps():
    """irk_set_tau rebuilds only the tau-dependent data: the reused handle gives the results of fresh
    handles for the new steps."""
    dim, N, k, Q = 3, 8, 3, 2
    stream = torch.cuda.Stream()
    with pkg.Group(dim, N, k, Q, [1e-3, 2e-3], stream=stream) as g:
        p = Problem(dim, N, k, Q, 1e-3)
        y0 = p.y0()
        ys = [torch.from_numpy(y0).cuda() for _ in range(2)]
        g.step_group(ys, [0.0, 0.0])
        new = [7e-3, 3e-4]
        g.set_tau(new)
        ys = [torch.from_numpy(y0).cuda() for _ in range(2)]
        per, _ = g.step_group(ys, [0.0, 0.0])
        assert per == [0, 0]
        got = [y.cpu().numpy() for y in ys]
    for r, tau in enumerate(new):
        alone, _ = _alone(dim, N, k, Q, tau, 0.0, y0, stream)
        assert np.abs(got[r] - alone).max() <= 1e-12 * np.abs(alone).max(), r


def test_one_failing_request_leaves_the_others_intact():
    """Host-side fault injection: a NaN in one request's y_n gives IRK_ENUMERIC for that request
    only; its y is unchanged and the other requests complete as alone."""
    dim, N, k, Q = 3, 6, 2, 3
    taus = [1e-3, 2e-3, 3e-3]
    stream = torch.cuda.Stream()
    p = Problem(dim, N, k, Q, 1e-3)
    y0 = p.y0()
    with pkg.Group(dim, N, k, Q, taus, stream=stream) as g:
        ys = [torch.from_numpy(y0).cuda() for _ in range(3)]
        idx = (2 * N + 1) ** 2 * 5 + (2 * N + 1) * 5 + 5
        ys[1][idx] = float("nan")
        bad = ys[1].clone()
        per, _ = g.step_group(ys, [0.0] * 3)
        assert per[1] == _capi.IRK_ENUMERIC and per[0] == 0 and per[2] == 0
        assert torch.equal(torch.nan_to_num(ys[1]), torch.nan_to_num(bad))
        got = [ys[0].cpu().numpy(), ys[2].cpu().numpy()]
    for r, i in ((0, 0), (1, 2)):
        alone, _ = _alone(dim, N, k, Q, taus[i], 0.0, y0, stream)
        assert np.abs(got[r] - alone).max() <= 1e-12 * np.abs(alone).max()


def test_float_float_group_equals_alone():
    """The float-float outer arithmetic (op_ff = 1) in a group: each request as alone."""
    dim, N, k, Q = 3, 8, 3, 2
    taus = [1e-3, 3e-3, 6e-4]
    stream = torch.cuda.Stream()
    y0 = Problem(dim, N, k, Q, 1e-3).y0()
    with pkg.Group(dim, N, k, Q, taus, stream=stream, op_ff=1) as g:
        ys = [torch.from_numpy(y0).cuda() for _ in taus]
        per, _ = g.step_group(ys, [0.0] * 3)
        assert per == [0, 0, 0]
        got = [y.cpu().numpy() for y in ys]
    for r, tau in enumerate(taus):
        with pkg.Solver(dim, N, k, Q, tau, stream=stream, op_ff=1) as s:
            y = torch.from_numpy(y0).cuda()
            s.step(y, 0.0)
            s.synchronize()
            alone = y.cpu().numpy()
        assert np.abs(got[r] - alone).max() <= 1e-12 * np.abs(alone).max(), r


def test_group_arguments():
    with pytest.raises(pkg.IrkError):
        pkg.Group(3, 8, 2, 9, [1e-3, 1e-3])               # R Q > 16
    with pytest.raises(pkg.IrkError):
        pkg.Group(3, 8, 2, 3, [1e-3, -1.0])               # tau <= 0
    with pytest.raises(pkg.IrkError):
        pkg.Group(3, 8, 2, 3, [1e-3, 1e-3], variant=pkg.IRK_VARIANT_DIAG)
    with pkg.Group(3, 4, 2, 2, [1e-3, 1e-3]) as g:
        with pytest.raises(pkg.IrkError):
            g.step(g.vector(), 0.0)                       # groups step with irk_step_group
