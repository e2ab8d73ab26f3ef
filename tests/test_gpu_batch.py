"""Batched persistent CG over lattices of different sizes: every lattice must
reach the tolerance (true residual recomputed by the oracle) and agree with
the single-lattice solver."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

LATTICES = [(4, 4, 4, 4), (2, 4, 6, 8), (6, 6, 6, 6), (4, 6, 2, 6), (8, 8, 8, 8)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def make_problem(ctx, dims, rep, seed):
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, seed)
    b = synth.gaussian_spinor(dims, nc, seed + 1)
    b[oracle.parity_mask(dims) == 1] = 0
    gauge = fields.pack_gauge(ctx, dims, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, dims, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(dims, rep, hr.HR_F64, hr.HR_EVEN)
    return q, b, gauge, bp, xp


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_batch_solves_every_lattice(ctx, rep):
    m0 = -0.2
    probs = [make_problem(ctx, d, rep, 300 + 10 * k) for k, d in enumerate(LATTICES)]
    opts = hr.hr_solver_default_opts()
    work = fields.empty_bytes(hr.hr_cg_batch_workspace_bytes(LATTICES, rep))
    rc, infos = hr.hr_cg_solve_batch(ctx, LATTICES, m0, rep, opts, [p[2] for p in probs],
                                     [p[3] for p in probs], [p[4] for p in probs], work)
    assert rc == hr.HR_OK
    nc = 2 if rep == hr.HR_FUND else 3
    for k, d in enumerate(LATTICES):
        q, b, gauge, bp, xp = probs[k]
        x = fields.unpack_spinor(ctx, d, rep, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
        L = oracle.expand_links(d, nc, q)
        res = np.linalg.norm(b - oracle.normal(d, L, m0, x)) / np.linalg.norm(b)
        assert res <= 1e-10, (d, res)
        assert abs(res - infos[k].true_rel_residual) <= 1e-11
        # the same lattice through the single-lattice solver
        x1 = fields.zeros_spinor(d, rep, hr.HR_F64, hr.HR_EVEN)
        w1 = fields.empty_bytes(hr.hr_cg_workspace_bytes(d, rep, opts))
        rc1, info1 = hr.hr_cg_solve(ctx, d, m0, rep, opts, gauge, bp, x1, w1)
        assert rc1 == hr.HR_OK
        assert abs(info1.iters - infos[k].iters) <= 1
        xs = fields.unpack_spinor(ctx, d, rep, hr.HR_F64, hr.HR_EVEN, x1).cpu().numpy()
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_batch_device_loop_matches_host_chunks(ctx, rep):
    """The one-launch batch (device WHILE loop) and the chunked batch (host
    check every 5 iterations) run the same arithmetic: identical solutions and
    iteration counts; with maxiter 7 both stop at exactly 7."""
    m0 = -0.2
    sols = []
    for check_every in (0, 5):
        probs = [make_problem(ctx, d, rep, 400 + 10 * k) for k, d in enumerate(LATTICES)]
        opts = hr.hr_solver_default_opts()
        opts.check_every = check_every
        work = fields.empty_bytes(hr.hr_cg_batch_workspace_bytes(LATTICES, rep))
        rc, infos = hr.hr_cg_solve_batch(ctx, LATTICES, m0, rep, opts, [p[2] for p in probs],
                                         [p[3] for p in probs], [p[4] for p in probs], work)
        assert rc == hr.HR_OK
        xs = [fields.unpack_spinor(ctx, d, rep, hr.HR_F64, hr.HR_EVEN, probs[k][4]).cpu().numpy()
              for k, d in enumerate(LATTICES)]
        sols.append(([i.iters for i in infos], xs))
        opts.maxiter = 7
        probs = [make_problem(ctx, d, rep, 400 + 10 * k) for k, d in enumerate(LATTICES)]
        rc, infos = hr.hr_cg_solve_batch(ctx, LATTICES, m0, rep, opts, [p[2] for p in probs],
                                         [p[3] for p in probs], [p[4] for p in probs], work)
        assert rc == hr.HR_ERR_NOT_CONVERGED
        assert all(i.iters == 7 for i in infos)
    assert sols[0][0] == sols[1][0]
    for a, b in zip(sols[0][1], sols[1][1]):
        assert np.array_equal(a, b)


def test_batch_argument_checks(ctx):
    opts = hr.hr_solver_default_opts()
    assert hr.hr_cg_batch_workspace_bytes([(4, 4, 4, 3)], hr.HR_FUND) == 0
    assert hr.hr_cg_batch_workspace_bytes([(4, 4, 4, 4)], hr.HR_ADJ_MAT) == 0
    probs = [make_problem(ctx, (4, 4, 4, 4), hr.HR_FUND, 5)]
    with pytest.raises(hr.HrError):
        hr.hr_cg_solve_batch(ctx, [(4, 4, 4, 4)], 0.0, hr.HR_FUND, opts, [probs[0][2]], [probs[0][3]],
                             [probs[0][4]], fields.empty_bytes(16))
    opts.inner_prec = hr.HR_F32
    work = fields.empty_bytes(hr.hr_cg_batch_workspace_bytes([(4, 4, 4, 4)], hr.HR_FUND))
    with pytest.raises(hr.HrError):
        hr.hr_cg_solve_batch(ctx, [(4, 4, 4, 4)], 0.0, hr.HR_FUND, opts, [probs[0][2]], [probs[0][3]],
                             [probs[0][4]], work)
