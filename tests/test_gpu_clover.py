"""Clover and exponential-clover operators on the GPU against the oracle
(oracle/clover.py, itself pinned in tests/test_oracle_clover.py).

Tolerances (relative L2): FP64 1e-13 (the field is built in FP64 and stored as
double-float pairs), FP32 1e-6, FP16 spinors 4e-3 (with the FP32 clover field);
solves to a true residual of 1e-10 recomputed by the oracle.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import clover as ocl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import fields, hr  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}
REPS = [hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT]
PRECS = [hr.HR_F64, hr.HR_F32, hr.HR_F16]
KINDS = [hr.HR_CLOVER_SW, hr.HR_CLOVER_EXP]
M0, CSW = -0.1, 1.3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def nc_of(rep):
    return 2 if rep == hr.HR_FUND else 3


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cprec(prec):
    return hr.HR_F64 if prec == hr.HR_F64 else hr.HR_F32


def setup(ctx, lat, rep, prec, kind, seed, m0=M0, csw=CSW, smear=False):
    q = synth.haar_links(lat, seed)
    if smear:
        q, _, _ = synth.ape_smear_to_plaquette(q, lat, 0.6)
    nc = nc_of(rep)
    L = oracle.expand_links(lat, nc, q)
    A = ocl.site_term(lat, L, m0, csw, kind)
    qd = fields.gauge_to_device(q)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, qd)
    clov = fields.build_clover(ctx, lat, rep, cprec(prec), kind, m0, csw, qd)
    return q, L, A, gauge, clov


@pytest.mark.parametrize("inverse", [0, 1])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_site_term_matches_oracle(ctx, rep, prec, kind, inverse):
    lat = (4, 6, 2, 6)
    nc = nc_of(rep)
    q, L, A, gauge, clov = setup(ctx, lat, rep, prec, kind, 11)
    psi = synth.gaussian_spinor(lat, nc, 12)
    dpsi = fields.spinor_to_device(psi)
    for par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(ctx, lat, rep, prec, par, dpsi)
        dst = fields.empty_spinor(lat, rep, prec, par)
        hr.hr_clover_apply(ctx, lat, rep, prec, par, inverse, 1, clov, src, dst)
        got = fields.unpack_spinor(ctx, lat, rep, prec, par, dst).cpu().numpy()
        m = oracle.parity_mask(lat) == par
        M = np.linalg.inv(A[m]) if inverse else A[m]
        want = ocl.apply_site(M, psi[m])
        assert rel(got[m], want) <= TOL[prec], (par, rel(got[m], want))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_full_operator_matches_oracle(ctx, rep, prec, kind):
    lat = hr.Lattice((4, 4, 4, 4), 1)
    nc = nc_of(rep)
    q, L, A, gauge, clov = setup(ctx, lat, rep, prec, kind, 21)
    psi = synth.gaussian_spinor(lat, nc, 22)
    src = fields.pack_spinor(ctx, lat, rep, prec, hr.HR_FULL, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, hr.HR_FULL)
    hr.hr_dirac_apply_clover(ctx, lat, rep, prec, gauge, clov, src, dst)
    got = fields.unpack_spinor(ctx, lat, rep, prec, hr.HR_FULL, dst).cpu().numpy()
    assert rel(got, ocl.dirac(lat, L, A, psi, bc=1)) <= TOL[prec]


@pytest.mark.parametrize("op", [hr.HR_OP_SCHUR, hr.HR_OP_SCHUR_DAG, hr.HR_OP_NORMAL])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_schur_operators_match_oracle(ctx, rep, prec, kind, op):
    lat = hr.Lattice((4, 6, 8, 10), 9)
    nc = nc_of(rep)
    q, L, A, gauge, clov = setup(ctx, lat, rep, prec, kind, 31)
    psi = synth.gaussian_spinor(lat, nc, 32)
    even = oracle.parity_mask(lat) == 0
    psi[~even] = 0
    src = fields.pack_spinor(ctx, lat, rep, prec, hr.HR_EVEN, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(lat, rep, prec, op))
    hr.hr_dirac_eo_clover(ctx, lat, rep, prec, hr.HR_EVEN, op, 1, gauge, clov, src, dst, work)
    got = fields.unpack_spinor(ctx, lat, rep, prec, hr.HR_EVEN, dst).cpu().numpy()
    if op == hr.HR_OP_NORMAL:
        want = ocl.normal(lat, L, A, psi, bc=9)
    else:
        want = ocl.schur(lat, L, A, psi, dagger=op == hr.HR_OP_SCHUR_DAG, bc=9)
    tol = TOL[prec] * (10 if prec != hr.HR_F16 else 2)
    assert rel(got[even], want[even]) <= tol


def _forced(tmp_path, monkeypatch, lat, rep, prec, variant, block, n_rhs=1):
    import json

    key = f"hop:r{rep}:p{prec}:{lat[0]}x{lat[1]}x{lat[2]}x{lat[3]}:n{n_rhs}"
    cache = tmp_path / f"cl_{rep}_{prec}_{variant}_{block}_{n_rhs}.json"
    cache.write_text(json.dumps({key: [variant, block]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    return hr.Context(0)


@pytest.mark.parametrize("variant", list(range(14)))
def test_clover_launches_do_not_depend_on_the_tuned_shape(tmp_path, monkeypatch, variant):
    """Clover launches run their own kernel instantiations whatever shape the
    tuner chose for the Wilson hop (fundamental FP64, exponential clover)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lat = (4, 6, 8, 10)
    c = _forced(tmp_path, monkeypatch, lat, hr.HR_FUND, hr.HR_F64, variant, 128)
    q, L, A, gauge, clov = setup(c, lat, hr.HR_FUND, hr.HR_F64, hr.HR_CLOVER_EXP, 41)
    psi = synth.gaussian_spinor(lat, 2, 42)
    even = oracle.parity_mask(lat) == 0
    psi[~even] = 0
    src = fields.pack_spinor(c, lat, 0, 0, hr.HR_EVEN, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, 0, 0, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(lat, 0, 0, hr.HR_OP_NORMAL))
    hr.hr_dirac_eo_clover(c, lat, 0, 0, hr.HR_EVEN, hr.HR_OP_NORMAL, 1, gauge, clov, src, dst, work)
    got = fields.unpack_spinor(c, lat, 0, 0, hr.HR_EVEN, dst).cpu().numpy()
    assert rel(got[even], ocl.normal(lat, L, A, psi)[even]) <= 1e-12


@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
def test_multi_rhs_equals_single(ctx, prec):
    lat = (4, 4, 6, 4)
    n = 4
    q, L, A, gauge, clov = setup(ctx, lat, hr.HR_FUND, prec, hr.HR_CLOVER_SW, 51)
    psis = synth.gaussian_spinor(lat, 2, 52, n_rhs=n)
    psis[:, oracle.parity_mask(lat) == 1] = 0
    src = fields.pack_spinor(ctx, lat, 0, prec, hr.HR_EVEN, fields.spinor_to_device(psis))
    dst = fields.empty_spinor(lat, 0, prec, hr.HR_EVEN, n)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(lat, 0, prec, hr.HR_OP_NORMAL, n))
    hr.hr_dirac_eo_clover(ctx, lat, 0, prec, hr.HR_EVEN, hr.HR_OP_NORMAL, n, gauge, clov, src, dst, work)
    got = fields.unpack_spinor(ctx, lat, 0, prec, hr.HR_EVEN, dst, n).cpu().numpy()
    even = oracle.parity_mask(lat) == 0
    for r in range(n):
        assert rel(got[r][even], ocl.normal(lat, L, A, psis[r])[even]) <= 10 * TOL[prec]


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_cg_true_residual(ctx, rep, kind, inner):
    lat = hr.Lattice((8, 4, 6, 4), 1)
    nc = nc_of(rep)
    q, L, A, gauge, clov = setup(ctx, lat, rep, hr.HR_F64, kind, 61, m0=-0.2, csw=1.0, smear=True)
    b = synth.gaussian_spinor(lat, nc, 62)
    b[oracle.parity_mask(lat) == 1] = 0
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(lat, rep, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_cg_clover_workspace_bytes(lat, rep, opts))
    rc, info = hr.hr_cg_solve_clover(ctx, lat, rep, opts, gauge, clov, bp, xp, work)
    assert rc == hr.HR_OK, info.true_rel_residual
    x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
    res = np.linalg.norm(b - ocl.normal(lat, L, A, x, bc=1)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert abs(res - info.true_rel_residual) <= 1e-11


@pytest.mark.parametrize("system", [hr.HR_SYSTEM_D, hr.HR_SYSTEM_DDAG_D])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_full_lattice_solve(ctx, rep, system):
    lat = (4, 4, 6, 4)
    nc = nc_of(rep)
    q, L, A, gauge, clov = setup(ctx, lat, rep, hr.HR_F64, hr.HR_CLOVER_SW, 71, m0=0.05, csw=1.0)
    b = synth.gaussian_spinor(lat, nc, 72)
    opts = hr.hr_solver_default_opts()
    opts.tol = 1e-11
    bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(b))
    xp = fields.empty_spinor(lat, rep, hr.HR_F64, hr.HR_FULL)
    work = fields.empty_bytes(hr.hr_solve_full_clover_workspace_bytes(lat, rep, opts, system))
    rc, info = hr.hr_solve_full_clover(ctx, lat, rep, opts, system, gauge, clov, bp, xp, work)
    assert rc == hr.HR_OK
    x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_FULL, xp).cpu().numpy()
    ax = ocl.dirac(lat, L, A, x)
    if system == hr.HR_SYSTEM_DDAG_D:
        ax = oracle.gamma5(ocl.dirac(lat, L, A, oracle.gamma5(ax)))
    res = np.linalg.norm(b - ax) / np.linalg.norm(b)
    assert res <= 1e-9, res
    assert abs(res - info.true_rel_residual) <= 1e-10


def test_argument_checks(ctx):
    lat = (4, 4, 4, 4)
    assert hr.hr_clover_packed_bytes(lat, hr.HR_FUND, hr.HR_F16) == 0
    assert hr.hr_clover_packed_bytes(lat, hr.HR_FUND, hr.HR_F64) > hr.hr_clover_packed_bytes(lat, hr.HR_FUND, hr.HR_F32)
    assert hr.hr_clover_packed_bytes(lat, hr.HR_ADJ, hr.HR_F64) == hr.hr_clover_packed_bytes(lat, hr.HR_ADJ_MAT, hr.HR_F64)
    qd = fields.gauge_to_device(synth.haar_links(lat, 81))
    out = fields.empty_bytes(hr.hr_clover_packed_bytes(lat, hr.HR_FUND, hr.HR_F64))
    with pytest.raises(hr.HrError):
        hr.hr_clover_build(ctx, lat, hr.HR_FUND, hr.HR_F64, 7, 0.0, 1.0, qd, out)
    with pytest.raises(hr.HrError):
        hr.hr_clover_build(ctx, lat, hr.HR_FUND, hr.HR_F16, hr.HR_CLOVER_SW, 0.0, 1.0, qd, out)
    opts = hr.hr_solver_default_opts()
    g = fields.pack_gauge(ctx, lat, 0, 0, qd)
    b = fields.zeros_spinor(lat, 0, 0, hr.HR_EVEN)
    x = fields.zeros_spinor(lat, 0, 0, hr.HR_EVEN)
    w = fields.empty_bytes(hr.hr_cg_clover_workspace_bytes(lat, 0, opts))
    with pytest.raises(hr.HrError):
        hr.hr_cg_solve_clover(ctx, lat, 0, opts, g, None, b, x, w)
