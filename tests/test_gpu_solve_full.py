"""Full-lattice solves through the even-odd reduction (source preparation,
Schur CG, odd reconstruction; D^+ D as two such solves), checked with the
FP64 oracle: the residual of the full system recomputed by the oracle from the
GPU's x, and agreement with the oracle's own even-odd solution."""

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


def solve(ctx, dims, rep, q, m0, b, system, inner=hr.HR_F64, tol=1e-11):
    opts = hr.hr_solver_default_opts()
    opts.tol = tol
    opts.inner_prec = inner
    gauge = fields.pack_gauge(ctx, dims, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, dims, rep, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(b))
    xp = fields.empty_spinor(dims, rep, hr.HR_F64, hr.HR_FULL)
    work = fields.empty_bytes(hr.hr_solve_full_workspace_bytes(dims, rep, opts, system))
    rc, info = hr.hr_solve_full(ctx, dims, m0, rep, opts, system, gauge, bp, xp, work)
    x = fields.unpack_spinor(ctx, dims, rep, hr.HR_F64, hr.HR_FULL, xp).cpu().numpy()
    return rc, info, x


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_solve_d_full_lattice(ctx, rep, inner):
    dims = (4, 4, 6, 4)
    m0 = 0.05
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, 501)
    b = synth.gaussian_spinor(dims, nc, 502)
    rc, info, x = solve(ctx, dims, rep, q, m0, b, hr.HR_SYSTEM_D, inner)
    assert rc == hr.HR_OK
    L = oracle.expand_links(dims, nc, q)
    res = np.linalg.norm(b - oracle.dirac(dims, L, m0, x)) / np.linalg.norm(b)
    assert res <= 1e-9, res
    assert abs(res - info.true_rel_residual) <= 1e-10
    # the oracle's own even-odd route: source, Schur CG, reconstruction
    bhat = oracle.eo_source(dims, L, m0, b)
    rhs = oracle.schur(dims, L, m0, bhat, dagger=True)
    xe, it, tr, ok = oracle.cg(dims, L, m0, rhs, tol=1e-12)
    xo = oracle.eo_reconstruct(dims, L, m0, b, xe)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-8


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_solve_ddag_d_full_lattice(ctx, rep):
    dims = (4, 4, 4, 6)
    m0 = 0.1
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, 511)
    b = synth.gaussian_spinor(dims, nc, 512)
    rc, info, x = solve(ctx, dims, rep, q, m0, b, hr.HR_SYSTEM_DDAG_D)
    assert rc == hr.HR_OK
    L = oracle.expand_links(dims, nc, q)
    dx = oracle.dirac(dims, L, m0, x)
    ddx = oracle.gamma5(oracle.dirac(dims, L, m0, oracle.gamma5(dx)))  # D^+ = g5 D g5
    res = np.linalg.norm(b - ddx) / np.linalg.norm(b)
    assert res <= 1e-9, res
    assert abs(res - info.true_rel_residual) <= 1e-10


def test_solve_full_argument_checks(ctx):
    dims = (4, 4, 4, 4)
    opts = hr.hr_solver_default_opts()
    assert hr.hr_solve_full_workspace_bytes(dims, hr.HR_FUND, opts, 7) == 0
    opts.n_rhs = 2
    assert hr.hr_solve_full_workspace_bytes(dims, hr.HR_FUND, opts, hr.HR_SYSTEM_D) == 0
