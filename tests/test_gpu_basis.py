"""The basis changes of Eq. (irk:P) around the block V-cycles (irk_basis_to_mg / irk_basis_from_mg)
and the float <-> double conversions they end and start with.

to_mg: b = S~^{-1} r, rounded to FP32 (nearest, ties to even).  S~ is unit lower triangular, so
stage 0 of b is stage 0 of r rounded alone: it must equal numpy's float32 cast bit for bit on
every class of value (exact ties to even and to odd, values either side of a tie, the largest
float and the values that round to infinity, results in and below the subnormal range, zeros of
both signs, infinities, NaN).  The other stages, whose FP64 sums the GPU and numpy may round
apart in the last bit, lie within one FP32 ulp of float32(S~^{-1} r), S~^{-1} the handle's own
factor (itself within 1e-12 of the oracle's, checked here too).
from_mg: z = S~ x from FP32 x: stage 0 of z is stage 0 of x widened, exactly (subnormal floats,
zeros, infinities, NaN included); the other stages within 1e-15 of S~ x in FP64.
Q = 3 runs the structured combination kernel, Q = 7 the general one; with the FP64 hierarchy the
multigrid side is FP64 and stage 0 passes through unchanged.
"""
import numpy as np
import pytest
import torch

import paper_2209_06700_gb300 as pkg
from oracle.tableau import lu_preconditioner_factors

pytestmark = pytest.mark.gpu

F32_MAX = float(np.finfo(np.float32).max)


def _special_doubles(n, rng):
    """n FP64 values covering the rounding cases of binary64 -> binary32."""
    f = rng.uniform(1.0, 2.0, n).astype(np.float32)
    f *= np.float32(2.0) ** rng.integers(-20, 20, n).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    tie = (f.astype(np.float64) + nxt.astype(np.float64)) / 2          # exact midpoints
    vals = [tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf),
            rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-160, 140, n)]  # wide exponents
    vals = np.concatenate(vals)
    vals *= np.where(rng.random(vals.size) < 0.5, -1.0, 1.0)
    edge = [0.0, -0.0, np.inf, -np.inf, np.nan, F32_MAX, -F32_MAX,
            F32_MAX + 2.0 ** 103, np.nextafter(F32_MAX + 2.0 ** 103, 0.0), 2.0 ** 128,
            2.0 ** -126, np.nextafter(2.0 ** -126, 0.0), 2.0 ** -149, 2.0 ** -150,
            np.nextafter(2.0 ** -150, 1.0), 3 * 2.0 ** -150, 2.0 ** -151, 1e-300, 5e-324,
            1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -50]
    out = np.concatenate([np.array(edge), vals])
    return np.resize(out, n)


def _special_floats(n, rng):
    """n FP32 values: normal over the whole range, subnormal, zeros, infinities, NaN."""
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, F32_MAX, 2.0 ** -126, 2.0 ** -149,
                     3 * 2.0 ** -149, 2.0 ** -127 + 2.0 ** -149], dtype=np.float32)
    out = bits.view(np.float32).copy()
    out[:edge.size] = edge
    return out


def _factors(s, Q):
    """The handle's S~ and S~^{-1}, after checking them against the oracle's (Eq. irk:P)."""
    F = lu_preconditioner_factors(Q)
    out = {}
    for name in ("S", "Sinv"):
        got = s.tableau(name)
        assert np.abs(got - F[name]).max() <= 1e-12 * max(1.0, np.abs(F[name]).max())
        out[name] = got
    return out


def _same_bits(got, ref):
    """Bit for bit, except that NaN matches any NaN and a zero either zero (the general
    combination kernel forms 1 * (-0) + 0 = +0 before converting)."""
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    it = np.uint32 if got.dtype == np.float32 else np.uint64
    same = (got.view(it) == ref.view(it)) | ((got == 0) & (ref == 0)) | nan
    assert same.all(), (got[~same][:5], ref[~same][:5])


@pytest.mark.parametrize("Q,mg", [(3, 32), (7, 32), (3, 64), (2, 0)])
def test_basis_to_mg(Q, mg):
    rng = np.random.default_rng(11 + Q)
    with pkg.Solver(3, 4, 2, Q, 1e-2, mg_precision=mg) as s:
        F = _factors(s, Q)
        n, stride = s.n, s.stride
        f32 = (mg == 32) or (mg == 0 and Q <= 5)
        mdt = torch.float32 if f32 else torch.float64
        # stage 0 alone: the conversion on every class of value
        r = np.zeros((Q, stride))
        r[0, :n] = _special_doubles(n, rng)
        rd = torch.from_numpy(r).cuda()
        b = torch.zeros(Q, stride, dtype=mdt, device="cuda")
        s.basis_to_mg(rd, b)
        s.synchronize()
        got0 = b[0, :n].cpu().numpy()
        with np.errstate(over="ignore", invalid="ignore"):
            ref0 = r[0, :n].astype(np.float32) if f32 else r[0, :n]
        _same_bits(got0, ref0)
        # every stage: S~^{-1} r
        r = rng.standard_normal((Q, stride)) * np.exp(rng.uniform(-20, 20, (Q, stride)))
        rd = torch.from_numpy(r).cuda()
        s.basis_to_mg(rd, b)
        s.synchronize()
        got = b[:, :n].double().cpu().numpy()
        exact = F["Sinv"] @ r[:, :n]
        if f32:
            ref = exact.astype(np.float32)
            # one FP32 ulp, plus the FP64 rounding of the sum where it cancels
            tol = np.spacing(np.abs(ref)).astype(np.float64) + 4e-16 * (np.abs(F["Sinv"]) @ np.abs(r[:, :n]))
            assert np.all(np.abs(got - ref) <= tol)
        else:
            assert np.all(np.abs(got - exact) <= 1e-15 * np.abs(F["Sinv"]) @ np.abs(r[:, :n]))


@pytest.mark.parametrize("Q,mg", [(3, 32), (7, 32), (3, 64)])
def test_basis_from_mg(Q, mg):
    rng = np.random.default_rng(21 + Q)
    with pkg.Solver(3, 4, 2, Q, 1e-2, mg_precision=mg) as s:
        F = _factors(s, Q)
        n, stride = s.n, s.stride
        f32 = mg == 32
        mdt = torch.float32 if f32 else torch.float64
        z = torch.zeros(Q, stride, dtype=torch.float64, device="cuda")
        if f32:
            x = np.zeros((Q, stride), dtype=np.float32)
            x[0, :n] = _special_floats(n, rng)
            s.basis_from_mg(torch.from_numpy(x).cuda(), z)
            s.synchronize()
            with np.errstate(invalid="ignore"):
                _same_bits(z[0, :n].cpu().numpy(), x[0, :n].astype(np.float64))
        x = rng.standard_normal((Q, stride)).astype(np.float32 if f32 else np.float64)
        s.basis_from_mg(torch.from_numpy(x).cuda().to(mdt), z)
        s.synchronize()
        got = z[:, :n].cpu().numpy()
        xs = x[:, :n].astype(np.float64)
        ref = F["S"] @ xs
        assert np.all(np.abs(got - ref) <= 1e-15 * (np.abs(F["S"]) @ np.abs(xs)))
        assert np.array_equal(got[0], xs[0])


def test_basis_arguments():
    with pkg.Solver(3, 4, 2, 3, 1e-2, variant=pkg.IRK_VARIANT_DIAG) as s:
        r = s.stage_vector()
        with pytest.raises(pkg.IrkError):
            s.basis_to_mg(r, s.stage_vector(dtype=torch.float32))
    with pkg.Group(3, 4, 2, 2, [1e-2, 2e-2]) as g:
        with pytest.raises(pkg.IrkError):
            g.basis_from_mg(g.stage_vector(dtype=torch.float32), g.stage_vector())
    with pkg.Solver(3, 4, 2, 3, 1e-2) as s:
        with pytest.raises(pkg.IrkError):
            s.basis_to_mg(s.stage_vector(), None)
