"""CG solves of Mhat^+ Mhat x = b on the GPU, checked with the FP64 oracle.

The pass criterion is the one the method fixes: the true residual
|b - A x| / |b| <= 1e-10, recomputed here by the oracle in FP64 from the GPU's
x.  The GPU solution is also compared with the oracle's own CG solution
(relative difference bounded by cond(A) * tol; reported, and gated loosely).
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


@pytest.fixture(scope="module")
def smeared_8():
    dims = (8, 8, 8, 8)
    q, steps, p = synth.ape_smear_to_plaquette(synth.haar_links(dims, 1002), dims, 0.6)
    return dims, q


def true_rel_residual(dims, L, m0, b, x):
    r = b - oracle.normal(dims, L, m0, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def run_solve(ctx, dims, rep, q, m0, b, inner, n_rhs=1, tol=1e-10, maxiter=20000, check_every=0, delta=None):
    opts = hr.hr_solver_default_opts()
    opts.check_every = check_every
    if delta is not None:
        opts.reliable_delta = delta
    opts.tol = tol
    opts.maxiter = maxiter
    opts.inner_prec = inner
    opts.n_rhs = n_rhs
    gauge = fields.pack_gauge(ctx, dims, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, dims, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(dims, rep, hr.HR_F64, hr.HR_EVEN, n_rhs)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(dims, rep, opts))
    rc, info = hr.hr_cg_solve(ctx, dims, m0, rep, opts, gauge, bp, xp, work)
    x = fields.unpack_spinor(ctx, dims, rep, hr.HR_F64, hr.HR_EVEN, xp, n_rhs).cpu().numpy()
    return rc, info, x


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_cg_true_residual(ctx, smeared_8, rep, inner):
    dims, q = smeared_8
    m0 = -0.2
    nc = 2 if rep == hr.HR_FUND else 3
    b = synth.gaussian_spinor(dims, nc, 2002)
    b[oracle.parity_mask(dims) == 1] = 0
    rc, info, x = run_solve(ctx, dims, rep, q, m0, b, inner)
    assert rc == hr.HR_OK, info.true_rel_residual
    L = oracle.expand_links(dims, nc, q)
    res = true_rel_residual(dims, L, m0, b, x)
    assert res <= 1e-10, res
    assert abs(res - info.true_rel_residual) <= 1e-11
    xo, it, tr, ok = oracle.cg(dims, L, m0, b, tol=1e-10)
    assert ok
    if inner == hr.HR_F64:
        assert abs(info.iters - it) <= 2, (info.iters, it)
    even = oracle.parity_mask(dims) == 0
    assert np.linalg.norm((x - xo)[even]) / np.linalg.norm(xo[even]) < 1e-7


def test_cg_multi_rhs_matches_single(ctx, smeared_8):
    dims, q = smeared_8
    m0 = -0.2
    n = 4
    bs = synth.gaussian_spinor(dims, 2, 3000, n_rhs=n)
    bs[:, oracle.parity_mask(dims) == 1] = 0
    rc, info, xs = run_solve(ctx, dims, hr.HR_FUND, q, m0, bs, hr.HR_F32, n_rhs=n)
    assert rc == hr.HR_OK
    L = oracle.expand_links(dims, 2, q)
    for r in range(n):
        assert true_rel_residual(dims, L, m0, bs[r], xs[r]) <= 1e-10


@pytest.mark.parametrize("n_rhs", [1, 4])
def test_cg_binary16_two_tier_updates(ctx, smeared_8, n_rhs):
    """Binary16 inner solves refresh the residual in FP32 between FP64 ones.
    With delta 1e-2 the recurrence asks for a reliable update at every 1e-2
    of reduction; only those at 1e-4 of the last FP64 residual and at
    convergence are FP64 (the ones n_reliable_updates counts): 3 for tol
    1e-10 with one right-hand side, where the FP32-inner solve, whose updates
    are all FP64, needs 5.  The oracle recomputes every true residual."""
    dims, q = smeared_8
    m0 = -0.2
    b = synth.gaussian_spinor(dims, 2, 2005, n_rhs=n_rhs)
    b[:, oracle.parity_mask(dims) == 1] = 0
    rb = b if n_rhs > 1 else b[0]
    rc16, i16, x16 = run_solve(ctx, dims, hr.HR_FUND, q, m0, rb, hr.HR_F16, n_rhs=n_rhs, delta=1e-2)
    rc32, i32, x32 = run_solve(ctx, dims, hr.HR_FUND, q, m0, rb, hr.HR_F32, n_rhs=n_rhs, delta=1e-2)
    assert rc16 == hr.HR_OK and rc32 == hr.HR_OK
    L = oracle.expand_links(dims, 2, q)
    xs16 = x16 if n_rhs > 1 else x16[None]
    for r in range(n_rhs):
        assert true_rel_residual(dims, L, m0, b[r], xs16[r]) <= 1e-10
    assert i32.n_reliable_updates >= 4, i32.n_reliable_updates
    assert i16.n_reliable_updates <= (3 if n_rhs == 1 else 4), i16.n_reliable_updates
    assert i16.n_reliable_updates < i32.n_reliable_updates


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
def test_cg_device_loop_matches_host_chunks(ctx, smeared_8, inner):
    """The one-launch solve (device WHILE loop, reliable update in an IF node)
    and the chunked solve (host check every 7 iterations, reliable update gated
    inside its kernels) run the same arithmetic: identical x and counts."""
    dims, q = smeared_8
    b = synth.gaussian_spinor(dims, 2, 2003)
    b[oracle.parity_mask(dims) == 1] = 0
    rc0, i0, x0 = run_solve(ctx, dims, hr.HR_FUND, q, -0.2, b, inner, check_every=0)
    rc1, i1, x1 = run_solve(ctx, dims, hr.HR_FUND, q, -0.2, b, inner, check_every=7)
    assert rc0 == hr.HR_OK and rc1 == hr.HR_OK
    assert i0.iters == i1.iters and i0.n_reliable_updates == i1.n_reliable_updates
    assert np.array_equal(x0, x1)
    assert i0.true_rel_residual == i1.true_rel_residual <= 1e-10


@pytest.mark.parametrize("check_every", [0, 4])
def test_cg_maxiter_is_exact(ctx, smeared_8, check_every):
    """The iteration cap stops the recurrence on the device, also inside a
    graph of 4 (or, device loop, 8) iterations that 9 does not divide."""
    dims, q = smeared_8
    b = synth.gaussian_spinor(dims, 2, 4001)
    b[oracle.parity_mask(dims) == 1] = 0
    rc, info, x = run_solve(ctx, dims, hr.HR_FUND, q, -0.2, b, hr.HR_F32, maxiter=9, check_every=check_every)
    assert rc == hr.HR_ERR_NOT_CONVERGED
    assert info.iters == 9


def test_cg_not_converged_status(ctx, smeared_8):
    dims, q = smeared_8
    b = synth.gaussian_spinor(dims, 2, 4000)
    b[oracle.parity_mask(dims) == 1] = 0
    rc, info, x = run_solve(ctx, dims, hr.HR_FUND, q, -0.2, b, hr.HR_F64, maxiter=5)
    assert rc == hr.HR_ERR_NOT_CONVERGED
    assert info.iters >= 5 and info.true_rel_residual > 1e-10


def test_cg_zero_source(ctx, smeared_8):
    dims, q = smeared_8
    b = np.zeros((int(np.prod(dims)), 4, 2), complex)
    rc, info, x = run_solve(ctx, dims, hr.HR_FUND, q, -0.2, b, hr.HR_F64)
    assert rc == hr.HR_OK and np.all(x == 0)
