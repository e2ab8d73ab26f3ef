"""Twisted fermion boundary conditions (``hr_lattice.theta``) on the GPU.

psi(x + L_mu mu) = e^{i theta_mu} psi(x): the library applies the phase in a
separate hop kernel (the twist cannot ride in the packed SU(2) links); the
oracle multiplies the neighbour value a hop fetches across the boundary by its
factor (its definition, pinned in tests/test_oracle_twist.py).  Every
operator, solver, link derivative, the clover operators and an HMC trajectory
are compared with the oracle at the tolerances of the periodic tests: FP64
1e-13, FP32 1e-6, FP16 storage 4e-3 relative L2; solves to a true residual of
1e-10.
"""

import json

import numpy as np
import pytest

import oracle
import synth
from oracle import clover as ocl
from oracle import hmc as ohmc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import autograd as ag  # noqa: E402
from paper_2411_18511_gb300 import fields, hr  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}
REPS = [hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT]
PRECS = [hr.HR_F64, hr.HR_F32, hr.HR_F16]
THETA = (0.7, -1.1, 2.5, 0.4)
THETA_T = (0.9, 0.0, 0.0, 0.0)  # time only


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


def even_mask(dims):
    return oracle.parity_mask(dims) == 0


def gpu_hop(ctx, lat, rep, prec, gauge, psi, out_par):
    src = fields.pack_spinor(ctx, lat, rep, prec, 1 - out_par, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, out_par)
    hr.hr_dirac_eo(ctx, lat, 0.1, rep, prec, out_par, hr.HR_OP_HOP, 1, gauge, src, dst)
    return fields.unpack_spinor(ctx, lat, rep, prec, out_par, dst).cpu().numpy()


def hop_error(ctx, lat, rep, prec, q, psi):
    nc = nc_of(rep)
    L = oracle.expand_links(lat, nc, q)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, fields.gauge_to_device(q))
    worst = 0.0
    for out_par in (hr.HR_EVEN, hr.HR_ODD):
        got = gpu_hop(ctx, lat, rep, prec, gauge, psi, out_par)
        m = oracle.parity_mask(lat) == out_par
        psi_in = psi.copy()
        psi_in[m] = 0
        want = -0.5 * oracle.hop(lat, L, psi_in, parity=out_par)
        worst = max(worst, rel(got[m], want[m]))
    return worst


@pytest.mark.parametrize("bc", [0, 9])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
@pytest.mark.parametrize("dims", [(6, 4, 2, 6), (4, 6, 8, 10)])
def test_hop_matches_oracle(ctx, dims, rep, prec, bc):
    lat = hr.Lattice(dims, bc, THETA)
    q = synth.haar_links(dims, 11)
    psi = synth.gaussian_spinor(dims, nc_of(rep), 12)
    assert hop_error(ctx, lat, rep, prec, q, psi) <= TOL[prec]
    # and the twist made a difference
    L = oracle.expand_links(dims, nc_of(rep), q)
    assert rel(oracle.hop(lat, L, psi), oracle.hop(dims, L, psi, bc=bc)) > 1e-2


@pytest.mark.parametrize("rep", REPS)
def test_pi_twist_is_the_antiperiodic_bit(ctx, rep):
    dims = (4, 6, 2, 6)
    q = synth.haar_links(dims, 13)
    psi = synth.gaussian_spinor(dims, nc_of(rep), 14)
    tw = hr.Lattice(dims, 0, (np.pi, 0.0, 0.0, 0.0))
    ap = hr.Lattice(dims, 1)
    for par in (hr.HR_EVEN, hr.HR_ODD):
        m = oracle.parity_mask(dims) == par
        a = gpu_hop(ctx, tw, rep, hr.HR_F64, fields.pack_gauge(ctx, tw, rep, hr.HR_F64, fields.gauge_to_device(q)),
                    psi, par)
        b = gpu_hop(ctx, ap, rep, hr.HR_F64, fields.pack_gauge(ctx, ap, rep, hr.HR_F64, fields.gauge_to_device(q)),
                    psi, par)
        assert rel(a[m], b[m]) <= 1e-14


def test_multi_rhs_hop_equals_single(ctx):
    lat = hr.Lattice((4, 6, 8, 10), 1, THETA)
    n = 4
    q = synth.haar_links(lat, 15)
    psis = synth.gaussian_spinor(lat, 2, 16, n_rhs=n)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_ODD, fields.spinor_to_device(psis))
    dst = fields.empty_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, n)
    hr.hr_dirac_eo(ctx, lat, 0.1, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, hr.HR_OP_HOP, n, gauge, src, dst)
    got = fields.unpack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, dst, n).cpu().numpy()
    for r in range(n):
        one = gpu_hop(ctx, lat, hr.HR_FUND, hr.HR_F64, gauge, psis[r], hr.HR_EVEN)
        m = even_mask(lat)
        np.testing.assert_array_equal(got[r][m], one[m])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_full_operator_matches_oracle(ctx, rep, prec):
    lat = hr.Lattice((4, 4, 4, 4), 1, THETA)
    nc = nc_of(rep)
    q = synth.haar_links(lat, 21)
    psi = synth.gaussian_spinor(lat, nc, 22)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, lat, rep, prec, hr.HR_FULL, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, hr.HR_FULL)
    hr.hr_dirac_apply(ctx, lat, 0.1, rep, prec, gauge, src, dst)
    got = fields.unpack_spinor(ctx, lat, rep, prec, hr.HR_FULL, dst).cpu().numpy()
    assert rel(got, oracle.dirac(lat, oracle.expand_links(lat, nc, q), 0.1, psi)) <= TOL[prec]


@pytest.mark.parametrize("op", [hr.HR_OP_SCHUR, hr.HR_OP_SCHUR_DAG, hr.HR_OP_NORMAL])
@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
@pytest.mark.parametrize("rep", REPS)
def test_schur_operators_match_oracle(ctx, rep, prec, op):
    lat = hr.Lattice((4, 6, 8, 10), 9, THETA)
    m0 = -0.2
    nc = nc_of(rep)
    q = synth.haar_links(lat, 31)
    psi = synth.gaussian_spinor(lat, nc, 32)
    even = even_mask(lat)
    psi[~even] = 0
    L = oracle.expand_links(lat, nc, q)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, lat, rep, prec, hr.HR_EVEN, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(lat, rep, prec, op))
    hr.hr_dirac_eo(ctx, lat, m0, rep, prec, hr.HR_EVEN, op, 1, gauge, src, dst, work)
    got = fields.unpack_spinor(ctx, lat, rep, prec, hr.HR_EVEN, dst).cpu().numpy()
    if op == hr.HR_OP_NORMAL:
        want = oracle.normal(lat, L, m0, psi)
    else:
        want = oracle.schur(lat, L, m0, psi, dagger=op == hr.HR_OP_SCHUR_DAG)
    assert rel(got[even], want[even]) <= 10 * TOL[prec]


@pytest.mark.parametrize("variant", [0, 3, 8, 11])
def test_tuned_shape_does_not_matter(tmp_path, monkeypatch, variant):
    """A twisted lattice runs the twisted kernel whatever variant the cache names."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lat = hr.Lattice((4, 6, 8, 10), 0, THETA)
    key = f"hop:r0:p0:{lat[0]}x{lat[1]}x{lat[2]}x{lat[3]}:n1"
    cache = tmp_path / f"tw_{variant}.json"
    cache.write_text(json.dumps({key: [variant, 128]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    c = hr.Context(0)
    assert hr.hr_tune_lookup(c, lat, hr.HR_FUND, hr.HR_F64)[0] == variant
    q = synth.haar_links(lat, 41)
    psi = synth.gaussian_spinor(lat, 2, 42)
    assert hop_error(c, lat, hr.HR_FUND, hr.HR_F64, q, psi) <= TOL[hr.HR_F64]


def run_cg(ctx, lat, rep, q, m0, b, inner, n_rhs=1, gauge=None, xp=None, work=None):
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    opts.n_rhs = n_rhs
    if gauge is None:
        gauge = fields.pack_gauge(ctx, lat, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    if xp is None:
        xp = fields.zeros_spinor(lat, rep, hr.HR_F64, hr.HR_EVEN, n_rhs)
    if work is None:
        work = fields.empty_bytes(hr.hr_cg_workspace_bytes(lat, rep, opts))
    rc, info = hr.hr_cg_solve(ctx, lat, m0, rep, opts, gauge, bp, xp, work)
    x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, xp, n_rhs).cpu().numpy()
    return rc, info, x


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_cg_true_residual(ctx, rep, inner):
    lat = hr.Lattice((8, 4, 6, 4), 1, THETA)
    m0 = -0.2
    nc = nc_of(rep)
    q = synth.haar_links(lat, 61)
    b = synth.gaussian_spinor(lat, nc, 62)
    b[~even_mask(lat)] = 0
    rc, info, x = run_cg(ctx, lat, rep, q, m0, b, inner)
    assert rc == hr.HR_OK
    L = oracle.expand_links(lat, nc, q)
    res = np.linalg.norm(b - oracle.normal(lat, L, m0, x)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert abs(res - info.true_rel_residual) <= 1e-11


def test_cg_multi_rhs(ctx):
    lat = hr.Lattice((6, 4, 4, 6), 9, THETA)
    m0 = -0.2
    n = 4
    q = synth.haar_links(lat, 71)
    bs = synth.gaussian_spinor(lat, 2, 72, n_rhs=n)
    bs[:, ~even_mask(lat)] = 0
    rc, info, xs = run_cg(ctx, lat, hr.HR_FUND, q, m0, bs, hr.HR_F32, n_rhs=n)
    assert rc == hr.HR_OK
    L = oracle.expand_links(lat, 2, q)
    for r in range(n):
        res = np.linalg.norm(bs[r] - oracle.normal(lat, L, m0, xs[r])) / np.linalg.norm(bs[r])
        assert res <= 1e-10, (r, res)


def test_solver_graph_is_not_shared_across_twists(ctx):
    """The same buffers solved untwisted, then twisted, then untwisted again: each
    solve runs its own operator (the instantiated CG graph is keyed by the twist)."""
    dims = (4, 4, 6, 4)
    m0 = -0.2
    q = synth.haar_links(dims, 75)
    b = synth.gaussian_spinor(dims, 2, 76)
    b[~even_mask(dims)] = 0
    L = oracle.expand_links(dims, 2, q)
    plain, tw = hr.Lattice(dims, 1), hr.Lattice(dims, 1, THETA)
    opts = hr.hr_solver_default_opts()
    gauge = fields.pack_gauge(ctx, plain, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    xp = fields.zeros_spinor(plain, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(plain, hr.HR_FUND, opts))
    for lat in (plain, tw, plain):
        xp.zero_()
        rc, info, x = run_cg(ctx, lat, hr.HR_FUND, q, m0, b, hr.HR_F64, gauge=gauge, xp=xp, work=work)
        assert rc == hr.HR_OK
        res = np.linalg.norm(b - oracle.normal(lat, L, m0, x)) / np.linalg.norm(b)
        assert res <= 1e-10, (lat, res)


def test_batch_rejects_twisted_lattices(ctx):
    lats = [hr.Lattice((4, 4, 4, 4), 1), hr.Lattice((4, 4, 4, 4), 1, THETA_T)]
    probs = []
    for k, lat in enumerate(lats):
        q = synth.haar_links(lat, 80 + k)
        b = synth.gaussian_spinor(lat, 2, 90 + k)
        gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
        bp = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
        probs.append((gauge, bp, fields.zeros_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)))
    opts = hr.hr_solver_default_opts()
    work = fields.empty_bytes(hr.hr_cg_batch_workspace_bytes(lats, hr.HR_FUND))
    with pytest.raises(hr.HrError, match="twisted"):
        hr.hr_cg_solve_batch(ctx, lats, -0.2, hr.HR_FUND, opts, [p[0] for p in probs], [p[1] for p in probs],
                             [p[2] for p in probs], work)


@pytest.mark.parametrize("bc", [0, 1])
def test_force_and_link_grad(ctx, bc):
    lat = hr.Lattice((4, 6, 2, 6), bc, THETA)
    q = synth.haar_links(lat, 101)
    a = synth.gaussian_spinor(lat, 2, 102)
    b = synth.gaussian_spinor(lat, 2, 103)
    L = oracle.expand_links(lat, 2, q)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    ap = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(a))
    bp = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(b))
    V = int(np.prod(lat))
    F = torch.zeros((4, V, 3), dtype=torch.float64, device="cuda")
    hr.hr_force(ctx, lat, gauge, ap, bp, 1.0, F)
    assert rel(F.cpu().numpy(), oracle.force(lat, L, a, b)) <= 1e-13
    G = torch.zeros((4, V, 4), dtype=torch.float64, device="cuda")
    hr.hr_link_grad(ctx, lat, ap, bp, 1.0, G)
    assert rel(G.cpu().numpy(), oracle.link_grad(lat, a, b)) <= 1e-13
    # the twist reaches the derivative
    assert rel(oracle.force(lat, L, a, b), oracle.force(lat, L, a, b, theta=(0, 0, 0, 0))) > 1e-3


@pytest.mark.parametrize("system", [hr.HR_SYSTEM_D, hr.HR_SYSTEM_DDAG_D])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_full_lattice_solve(ctx, rep, system):
    lat = hr.Lattice((4, 4, 6, 4), 1, THETA)
    m0 = 0.05
    nc = nc_of(rep)
    q = synth.haar_links(lat, 111)
    b = synth.gaussian_spinor(lat, nc, 112)
    opts = hr.hr_solver_default_opts()
    opts.tol = 1e-11
    gauge = fields.pack_gauge(ctx, lat, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(b))
    xp = fields.empty_spinor(lat, rep, hr.HR_F64, hr.HR_FULL)
    work = fields.empty_bytes(hr.hr_solve_full_workspace_bytes(lat, rep, opts, system))
    rc, info = hr.hr_solve_full(ctx, lat, m0, rep, opts, system, gauge, bp, xp, work)
    assert rc == hr.HR_OK
    x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_FULL, xp).cpu().numpy()
    L = oracle.expand_links(lat, nc, q)
    Dx = oracle.dirac(lat, L, m0, x)
    if system == hr.HR_SYSTEM_DDAG_D:
        Dx = oracle.gamma5(oracle.dirac(lat, L, m0, oracle.gamma5(Dx)))
    res = np.linalg.norm(b - Dx) / np.linalg.norm(b)
    assert res <= 1e-9, res


def test_autograd_dirac_apply(ctx):
    lat = hr.Lattice((4, 6, 2, 6), 1, THETA)
    m0 = 0.1
    q = synth.haar_links(lat, 121)
    psi = synth.gaussian_spinor(lat, 2, 122)
    g = synth.gaussian_spinor(lat, 2, 123)
    qt = torch.tensor(q, device="cuda", requires_grad=True)
    pt = torch.tensor(psi, device="cuda", requires_grad=True)
    y = ag.DiracApply.apply(qt, pt, lat, m0)
    L = oracle.expand_links(lat, 2, q)
    assert rel(y.detach().cpu().numpy(), oracle.dirac(lat, L, m0, psi)) <= 1e-13
    y.backward(torch.tensor(g, device="cuda"))
    want_psi = oracle.gamma5(oracle.dirac(lat, L, m0, oracle.gamma5(g)))
    assert rel(pt.grad.cpu().numpy(), want_psi) <= 1e-13
    assert rel(qt.grad.cpu().numpy(), -0.5 * oracle.link_grad(lat, g, psi)) <= 1e-13


@pytest.mark.parametrize("op", [hr.HR_OP_SCHUR, hr.HR_OP_NORMAL])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_clover_schur_operators(ctx, rep, prec, op):
    lat = hr.Lattice((4, 6, 8, 10), 9, THETA)
    m0, csw = -0.2, 1.0
    nc = nc_of(rep)
    q = synth.haar_links(lat, 131)
    L = oracle.expand_links(lat, nc, q)
    A = ocl.site_term(lat, L, m0, csw, ocl.KIND_SW)
    qd = fields.gauge_to_device(q)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, qd)
    cp = hr.HR_F64 if prec == hr.HR_F64 else hr.HR_F32
    clov = fields.build_clover(ctx, lat, rep, cp, hr.HR_CLOVER_SW, m0, csw, qd)
    psi = synth.gaussian_spinor(lat, nc, 132)
    even = even_mask(lat)
    psi[~even] = 0
    src = fields.pack_spinor(ctx, lat, rep, prec, hr.HR_EVEN, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(lat, rep, prec, op))
    hr.hr_dirac_eo_clover(ctx, lat, rep, prec, hr.HR_EVEN, op, 1, gauge, clov, src, dst, work)
    got = fields.unpack_spinor(ctx, lat, rep, prec, hr.HR_EVEN, dst).cpu().numpy()
    want = ocl.normal(lat, L, A, psi) if op == hr.HR_OP_NORMAL else ocl.schur(lat, L, A, psi)
    tol = TOL[prec] * (10 if prec != hr.HR_F16 else 2)
    assert rel(got[even], want[even]) <= tol


def test_clover_cg(ctx):
    lat = hr.Lattice((8, 4, 6, 4), 1, THETA)
    m0, csw = -0.2, 1.0
    q = synth.haar_links(lat, 141)
    L = oracle.expand_links(lat, 2, q)
    A = ocl.site_term(lat, L, m0, csw, ocl.KIND_EXP)
    qd = fields.gauge_to_device(q)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, qd)
    clov = fields.build_clover(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_CLOVER_EXP, m0, csw, qd)
    b = synth.gaussian_spinor(lat, 2, 142)
    b[~even_mask(lat)] = 0
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = hr.HR_F16
    opts.reliable_delta = 0.01
    bp = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_cg_clover_workspace_bytes(lat, hr.HR_FUND, opts))
    rc, info = hr.hr_cg_solve_clover(ctx, lat, hr.HR_FUND, opts, gauge, clov, bp, xp, work)
    assert rc == hr.HR_OK
    x = fields.unpack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
    res = np.linalg.norm(b - ocl.normal(lat, L, A, x)) / np.linalg.norm(b)
    assert res <= 1e-10, res


def test_hmc_trajectory_matches_oracle(ctx):
    lat = hr.Lattice((4, 2, 2, 4), 1, THETA)
    beta, m0 = 2.2, 0.1
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(lat, 151), lat, 0.6)
    p = np.random.default_rng(152).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 3, 0.3, hr.HR_INTEGRATOR_OMELYAN)
    prm.solver.tol = 1e-13
    eta = synth.gaussian_spinor(lat, 2, 153) / np.sqrt(2.0)
    eta[oracle.parity_mask(lat) == 1] = 0
    eta_p = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(eta))
    qd = torch.tensor(q, device="cuda")
    pd = torch.tensor(p, device="cuda")
    work = fields.empty_bytes(hr.hr_hmc_workspace_bytes(lat, prm))
    info = hr.hr_hmc_trajectory(ctx, lat, prm, qd, pd, eta_p, work)
    ferm = ohmc.Fermions(lat, m0, eta, bc=1)
    qo, po, io = ohmc.trajectory(lat, q, p, beta, 3, 0.3, hr.HR_INTEGRATOR_OMELYAN, ferm)
    assert np.abs(qd.cpu().numpy() - qo).max() <= 1e-11
    assert np.abs(pd.cpu().numpy() - po).max() <= 1e-9
    assert abs(info.dH - io["dH"]) <= 1e-9
    assert abs(info.fermion_action_end - io["end"]["fermion"]) <= 1e-9
    # the twisted fermions moved the links differently from the untwisted ones
    qu, _, _ = ohmc.trajectory(lat, q, p, beta, 3, 0.3, hr.HR_INTEGRATOR_OMELYAN,
                               ohmc.Fermions(lat, m0, eta, bc=1, theta=(0, 0, 0, 0)))
    assert np.abs(qu - qo).max() > 1e-6


def test_non_finite_theta_is_rejected(ctx):
    lat = hr.Lattice((4, 4, 4, 4), 0, (0.1, float("nan"), 0.0, 0.0))
    q = synth.haar_links(lat, 161)
    gauge = fields.pack_gauge(ctx, hr.Lattice((4, 4, 4, 4)), hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    src = fields.zeros_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_ODD)
    dst = fields.empty_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    with pytest.raises(hr.HrError, match="theta"):
        hr.hr_dirac_eo(ctx, lat, 0.1, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, hr.HR_OP_HOP, 1, gauge, src, dst)


def test_tuner_skips_twisted_lattices(ctx):
    """Tuning a twisted lattice times nothing and keeps the untwisted choice of the extents."""
    dims = (4, 6, 8, 10)
    plain, tw = hr.Lattice(dims), hr.Lattice(dims, 0, THETA)
    q = synth.haar_links(dims, 171)
    psi = fields.spinor_to_device(synth.gaussian_spinor(dims, 2, 172))
    gauge = fields.pack_gauge(ctx, plain, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, plain, hr.HR_FUND, hr.HR_F64, hr.HR_ODD, psi)
    dst = fields.empty_spinor(plain, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    before = hr.hr_tune_lookup(ctx, plain, hr.HR_FUND, hr.HR_F64)
    res = hr.hr_autotune_hop(ctx, tw, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1, gauge, src, dst, reps=2)
    assert res.candidates == 0
    assert hr.hr_tune_lookup(ctx, plain, hr.HR_FUND, hr.HR_F64) == before


def test_full_size_48_sampled_sites(ctx):
    """48^4 fundamental FP64 twisted hop (time antiperiodic, all four directions
    twisted), checked on 2000 sampled output sites, half of them on boundary
    slices, against the oracle."""
    dims = (48, 48, 48, 48)
    lat = hr.Lattice(dims, 1, THETA)
    rep, prec = hr.HR_FUND, hr.HR_F64
    q = synth.haar_links(dims, 1013)
    psi = synth.gaussian_spinor(dims, 2, 2013)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, fields.gauge_to_device(q))
    dpsi = fields.spinor_to_device(psi)
    L = oracle.expand_links(dims, 2, q)
    x = np.indices(dims).reshape(4, -1).T
    edge = np.any((x == 0) | (x == np.array(dims) - 1), axis=1)
    rng = np.random.default_rng(17)
    for out_par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(ctx, lat, rep, prec, 1 - out_par, dpsi)
        dst = fields.empty_spinor(lat, rep, prec, out_par)
        hr.hr_dirac_eo(ctx, lat, 0.0, rep, prec, out_par, hr.HR_OP_HOP, 1, gauge, src, dst)
        got = fields.unpack_spinor(ctx, lat, rep, prec, out_par, dst).cpu().numpy()
        par = oracle.parity_mask(dims) == out_par
        on_edge = np.where(par & edge)[0]
        inside = np.where(par & ~edge)[0]
        sites = np.concatenate([rng.choice(on_edge, 1000, replace=False), rng.choice(inside, 1000, replace=False)])
        psi_in = psi.copy()
        psi_in[par] = 0
        want = -0.5 * oracle.hop_sites(lat, L, psi_in, sites)
        assert rel(got[sites], want) <= 1e-13
    del L
