"""HMC molecular dynamics on the GPU against the oracle (oracle/hmc.py, pinned in
tests/test_oracle_hmc.py): gauge force and action, link and momentum updates,
kinetic energy, and whole leapfrog / Omelyan trajectories with and without the
pseudofermion (same inputs; CG to 1e-13 on both sides), reversibility, and the
Markov chain driver."""

import numpy as np
import pytest

import oracle
import synth
from oracle import hmc as ohmc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import fields, hr  # noqa: E402
from paper_2411_18511_gb300.hmc import HMC  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def smeared(dims, seed):
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, seed), dims, 0.6)
    return q


@pytest.mark.parametrize("dims", [(4, 6, 2, 4), (8, 4, 4, 6)])
def test_gauge_force_and_action(ctx, dims):
    beta = 2.3
    q = synth.haar_links(dims, 11)
    F = torch.zeros((4, int(np.prod(dims)), 3), dtype=torch.float64, device="cuda")
    hr.hr_gauge_force(ctx, dims, beta, dev(q), 1.0, F)
    want = ohmc.gauge_force(dims, q, beta)
    assert rel(F.cpu().numpy(), want) <= 1e-13
    hr.hr_gauge_force(ctx, dims, beta, dev(q), -0.5, F)  # accumulates
    assert rel(F.cpu().numpy(), 0.5 * want) <= 1e-13
    S = hr.hr_gauge_action(ctx, dims, beta, dev(q))
    assert abs(S - ohmc.gauge_action(dims, q, beta)) <= 1e-12 * abs(S)


def test_updates_and_kinetic_energy(ctx):
    dims = (4, 4, 2, 6)
    V = int(np.prod(dims))
    q = synth.haar_links(dims, 21)
    p = np.random.default_rng(22).normal(size=(4, V, 3))
    F = np.random.default_rng(23).normal(size=(4, V, 3))
    qd, pd = dev(q), dev(p)
    hr.hr_link_update(ctx, dims, 0.37, pd, qd)
    np.testing.assert_allclose(qd.cpu().numpy(), ohmc.link_update(q, p, 0.37), atol=1e-14)
    hr.hr_mom_update(ctx, dims, 0.25, dev(F), pd)
    np.testing.assert_allclose(pd.cpu().numpy(), p - 0.25 * F, atol=1e-15)
    K = hr.hr_kinetic_energy(ctx, dims, pd)
    assert abs(K - ohmc.kinetic(p - 0.25 * F)) <= 1e-12 * K


def eta_field(ctx, lat, m0, seed):
    """A Gaussian even pseudofermion (full-lattice array) and its packed form."""
    eta = synth.gaussian_spinor(lat, 2, seed) / np.sqrt(2.0)
    eta[oracle.parity_mask(lat) == 1] = 0
    packed = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(eta))
    return eta, packed


def run_gpu(ctx, lat, q, p, prm, eta_packed, phi_packed=None):
    qd, pd = dev(q), dev(p)
    work = fields.empty_bytes(hr.hr_hmc_workspace_bytes(lat, prm))
    info = hr.hr_hmc_trajectory(ctx, lat, prm, qd, pd, eta_packed, work, phi=phi_packed)
    return qd.cpu().numpy(), pd.cpu().numpy(), info


@pytest.mark.parametrize("integrator", [hr.HR_INTEGRATOR_LEAPFROG, hr.HR_INTEGRATOR_OMELYAN])
@pytest.mark.parametrize("fermions", [False, True])
def test_trajectory_matches_oracle(ctx, integrator, fermions):
    lat = hr.Lattice((4, 2, 2, 4), 1)
    beta, m0 = 2.2, 0.1
    q = smeared(lat, 31)
    p = np.random.default_rng(32).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, fermions, 3, 0.3, integrator)
    prm.solver.tol = 1e-13
    eta, eta_p = eta_field(ctx, lat, m0, 33)
    qg, pg, info = run_gpu(ctx, lat, q, p, prm, eta_p if fermions else None)
    ferm = ohmc.Fermions(lat, m0, eta, bc=1) if fermions else None
    qo, po, io = ohmc.trajectory(lat, q, p, beta, 3, 0.3, integrator, ferm)
    assert np.abs(qg - qo).max() <= 1e-11
    assert np.abs(pg - po).max() <= 1e-9
    assert abs(info.dH - io["dH"]) <= 1e-9, (info.dH, io["dH"])
    assert abs(info.gauge_action_end - io["end"]["gauge"]) <= 1e-9
    assert abs(info.kinetic_end - io["end"]["kinetic"]) <= 1e-9
    if fermions:
        assert abs(info.fermion_action_end - io["end"]["fermion"]) <= 1e-9
        assert info.solves >= 4 and info.cg_iters > 0
    assert np.abs(qg - q).max() > 1e-3


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F16])
def test_trajectory_is_reversible(ctx, inner):
    lat = hr.Lattice((8, 8, 4, 4), 1)
    beta, m0 = 2.2, 0.05
    q = smeared(lat, 41)
    p = np.random.default_rng(42).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 5, 0.5, hr.HR_INTEGRATOR_OMELYAN)
    prm.solver.tol = 1e-12
    prm.solver.inner_prec = inner
    _, eta_p = eta_field(ctx, lat, m0, 43)
    q1, p1, i1 = run_gpu(ctx, lat, q, p, prm, eta_p)
    q2, p2, i2 = run_gpu(ctx, lat, q1, -p1, prm, eta_p)
    assert np.abs(q2 - q).max() <= 1e-9
    assert np.abs(p2 + p).max() <= 1e-7
    assert abs(i1.dH + i2.dH) <= 1e-7
    assert abs(i1.dH) < 1.0


def test_markov_chain(ctx):
    lat = hr.Lattice((4, 4, 4, 4), 1)
    q = dev(smeared(lat, 51))
    chain = HMC(ctx, lat, beta=2.2, m0=0.1, fermions=True, n_steps=8, tau=0.5, seed=52)
    plaq = []
    for _ in range(4):
        acc, info = chain.step(q)
        assert np.isfinite(info.dH) and abs(info.dH) < 2.0
        plaq.append(info.plaquette if acc else None)
    assert chain.accepted >= 2
    np.testing.assert_allclose(np.linalg.norm(q.cpu().numpy(), axis=-1), 1.0, atol=1e-13)


def test_argument_checks(ctx):
    lat = (4, 4, 4, 4)
    prm = hr.hr_hmc_params_default(2.0, 0.1, True, 0, 1.0)
    assert hr.hr_hmc_workspace_bytes(lat, prm) > 0
    q = dev(synth.identity_links(lat))
    p = torch.zeros((4, 256, 3), dtype=torch.float64, device="cuda")
    work = fields.empty_bytes(hr.hr_hmc_workspace_bytes(lat, prm))
    with pytest.raises(hr.HrError):
        hr.hr_hmc_trajectory(ctx, lat, prm, q, p, None, work)  # n_steps = 0
    prm.n_steps = 2
    with pytest.raises(hr.HrError):
        hr.hr_hmc_trajectory(ctx, lat, prm, q, p, None, work)  # fermions without eta
    prm.hasenbusch, prm.m0_hasenbusch = 1, 0.5
    eta = fields.zeros_spinor(lat, 0, 0, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_hmc_workspace_bytes(lat, prm))
    with pytest.raises(hr.HrError):
        hr.hr_hmc_trajectory(ctx, lat, prm, q, p, eta, work)  # Hasenbusch without phi


# ---------------------------------------------------------------- Hasenbusch

@pytest.mark.parametrize("integrator", [hr.HR_INTEGRATOR_LEAPFROG, hr.HR_INTEGRATOR_OMELYAN])
def test_hasenbusch_trajectory_matches_oracle(ctx, integrator):
    lat = hr.Lattice((4, 2, 2, 4), 1)
    beta, m0, mh = 2.2, 0.05, 0.5
    q = smeared(lat, 61)
    p = np.random.default_rng(62).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 3, 0.3, integrator)
    prm.hasenbusch, prm.m0_hasenbusch = 1, mh
    prm.solver.tol = 1e-13
    eta, eta_p = eta_field(ctx, lat, m0, 63)
    phi, phi_p = eta_field(ctx, lat, m0, 64)
    qg, pg, info = run_gpu(ctx, lat, q, p, prm, eta_p, phi_p)
    ferm = ohmc.Hasenbusch(lat, m0, mh, eta, phi, bc=1)
    qo, po, io = ohmc.trajectory(lat, q, p, beta, 3, 0.3, integrator, ferm)
    assert np.abs(qg - qo).max() <= 1e-11
    assert np.abs(pg - po).max() <= 1e-9
    assert abs(info.dH - io["dH"]) <= 1e-9, (info.dH, io["dH"])
    assert abs(info.fermion_action_end - io["end"]["fermion"]) <= 1e-9
    assert info.solves >= 8


def test_hasenbusch_heat_bath_and_chain(ctx):
    """The driver's two pseudofermions give S_f = |xi1|^2 + |xi2|^2 before the first
    step (checked with fields drawn the driver's way from known xi), and a short
    chain with Hasenbusch accepts."""
    lat = hr.Lattice((4, 4, 4, 4), 1)
    m0, mh = 0.05, 0.5
    q = dev(smeared(lat, 71))
    chain = HMC(ctx, lat, beta=2.2, m0=m0, fermions=True, n_steps=6, tau=0.5, seed=72, m0_hasenbusch=mh)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, q)
    rng = np.random.default_rng(73)
    xis = []
    for _ in range(2):
        xi = (rng.normal(size=(int(np.prod(lat)), 4, 2)) + 1j * rng.normal(size=(int(np.prod(lat)), 4, 2))) / np.sqrt(2)
        xi[oracle.parity_mask(lat) == 1] = 0
        xis.append(xi)
    packed = [fields.pack_spinor(ctx, lat, 0, 0, hr.HR_EVEN, fields.spinor_to_device(x)) for x in xis]
    eta = chain._schur(gauge, mh, packed[0], True)
    rhs = chain._schur(gauge, m0, packed[1], True)
    opts = hr.hr_solver_default_opts()
    opts.tol = 1e-13
    y = fields.zeros_spinor(lat, 0, 0, hr.HR_EVEN)
    hr.hr_cg_solve(ctx, lat, mh, 0, opts, gauge, rhs, y, fields.empty_bytes(hr.hr_cg_workspace_bytes(lat, 0, opts)))
    phi = chain._schur(gauge, mh, y, False)
    p = torch.zeros((4, int(np.prod(lat)), 3), dtype=torch.float64, device="cuda")
    prm = hr.hr_hmc_params_default(2.2, m0, True, 1, 1e-6)
    prm.hasenbusch, prm.m0_hasenbusch = 1, mh
    prm.solver.tol = 1e-13
    info = hr.hr_hmc_trajectory(ctx, lat, prm, q.clone(), p, eta, chain.work, phi=phi)
    want = sum(float(np.vdot(x, x).real) for x in xis)
    assert abs(info.fermion_action_start - want) <= 1e-9 * want
    for _ in range(3):
        acc, info = chain.step(q)
        assert np.isfinite(info.dH) and abs(info.dH) < 2.0
    assert chain.accepted >= 2


@pytest.mark.parametrize("hasenbusch", [None, 0.4])
def test_creutz_equality(ctx, hasenbusch):
    """<exp(-dH)> = 1 over an equilibrium chain: a consequence of the MD being
    reversible and area-preserving and of the heat baths drawing momenta and
    pseudofermions from exp(-H), so it tests the whole update at once
    (deterministic seeds; 4 standard errors of the mean)."""
    lat = hr.Lattice((4, 4, 4, 4), 1)
    q = dev(smeared(lat, 81))
    chain = HMC(ctx, lat, beta=2.2, m0=0.1, fermions=True, n_steps=6, tau=0.5, seed=82,
                m0_hasenbusch=hasenbusch)
    for _ in range(40):
        chain.step(q)
    w = []
    for _ in range(200):
        acc, info = chain.step(q)
        w.append(np.exp(-info.dH))
    w = np.array(w)
    err = w.std(ddof=1) / np.sqrt(len(w))
    assert abs(w.mean() - 1.0) <= 4 * err + 1e-3, (w.mean(), err)
    assert chain.accepted > 0.7 * chain.trajectories


@pytest.mark.parametrize("hasenbusch", [False, True])
@pytest.mark.parametrize("integrator", [hr.HR_INTEGRATOR_LEAPFROG, hr.HR_INTEGRATOR_OMELYAN])
def test_two_time_scales_match_oracle(ctx, integrator, hasenbusch):
    """n_steps_gauge = 3: the pseudofermion force on the outer level, three gauge
    steps per outer link update, against the oracle's nested integrator."""
    lat = hr.Lattice((4, 2, 2, 4), 1)
    beta, m0, mh = 2.2, 0.1, 0.6
    q = smeared(lat, 91)
    p = np.random.default_rng(92).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 2, 0.3, integrator)
    prm.solver.tol = 1e-13
    prm.n_steps_gauge = 3
    eta, eta_p = eta_field(ctx, lat, m0, 93)
    phi = phi_p = None
    if hasenbusch:
        prm.hasenbusch, prm.m0_hasenbusch = 1, mh
        phi, phi_p = eta_field(ctx, lat, m0, 94)
    qg, pg, info = run_gpu(ctx, lat, q, p, prm, eta_p, phi_p)
    ferm = ohmc.Hasenbusch(lat, m0, mh, eta, phi, bc=1) if hasenbusch else ohmc.Fermions(lat, m0, eta, bc=1)
    qo, po, io = ohmc.trajectory(lat, q, p, beta, 2, 0.3, integrator, ferm, n_steps_gauge=3)
    assert np.abs(qg - qo).max() <= 1e-11
    assert np.abs(pg - po).max() <= 1e-9
    assert abs(info.dH - io["dH"]) <= 1e-9, (info.dH, io["dH"])
    # and it is not the one-scale trajectory
    q1, _, _ = ohmc.trajectory(lat, q, p, beta, 2, 0.3, integrator, ferm)
    assert np.abs(q1 - qo).max() > 1e-8


def test_two_time_scales_reversible(ctx):
    lat = hr.Lattice((8, 8, 4, 4), 1)
    beta, m0 = 2.2, 0.05
    q = smeared(lat, 95)
    p = np.random.default_rng(96).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 3, 0.5, hr.HR_INTEGRATOR_OMELYAN)
    prm.solver.tol = 1e-12
    prm.n_steps_gauge = 4
    _, eta_p = eta_field(ctx, lat, m0, 97)
    q1, p1, i1 = run_gpu(ctx, lat, q, p, prm, eta_p)
    q2, p2, i2 = run_gpu(ctx, lat, q1, -p1, prm, eta_p)
    assert np.abs(q2 - q).max() <= 1e-9
    assert np.abs(p2 + p).max() <= 1e-7
    assert abs(i1.dH + i2.dH) <= 1e-7
    prm.n_steps_gauge = -1
    with pytest.raises(hr.HrError):
        run_gpu(ctx, lat, q, p, prm, eta_p)


@pytest.mark.parametrize("kind", [hr.HR_CLOVER_SW, hr.HR_CLOVER_EXP])
@pytest.mark.parametrize("m", [1, 3])
@pytest.mark.parametrize("integrator", [hr.HR_INTEGRATOR_LEAPFROG, hr.HR_INTEGRATOR_OMELYAN])
def test_clover_trajectory_matches_oracle(ctx, integrator, m, kind):
    """Clover (SW) fermions: the clover field rebuilt after every link update,
    S_f with -2 log det A_oo, the force of hops, site term and det term, on one
    or two time scales, against the oracle's CloverFermions."""
    from oracle import clover as ocl

    lat = hr.Lattice((4, 2, 2, 4), 1)
    beta, m0, csw = 2.2, 0.1, 1.1
    q = smeared(lat, 101)
    p = np.random.default_rng(102).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 2, 0.3, integrator)
    prm.solver.tol = 1e-13
    prm.n_steps_gauge = m
    prm.clover, prm.c_sw, prm.clover_kind = 1, csw, kind
    eta, eta_p = eta_field(ctx, lat, m0, 103)
    qg, pg, info = run_gpu(ctx, lat, q, p, prm, eta_p)
    ferm = ocl.CloverFermions(lat, m0, csw, eta, bc=1, kind=ocl.KIND_EXP if kind == hr.HR_CLOVER_EXP else ocl.KIND_SW)
    qo, po, io = ohmc.trajectory(lat, q, p, beta, 2, 0.3, integrator, ferm, n_steps_gauge=m)
    assert np.abs(qg - qo).max() <= 1e-11
    assert np.abs(pg - po).max() <= 1e-9
    assert abs(info.dH - io["dH"]) <= 1e-9, (info.dH, io["dH"])
    assert abs(info.fermion_action_start - io["start"]["fermion"]) <= 1e-9 * abs(io["start"]["fermion"])
    assert abs(info.fermion_action_end - io["end"]["fermion"]) <= 1e-9 * abs(io["end"]["fermion"])


def test_clover_chain(ctx):
    """The chain with clover fermions: eta = Mhat^+ xi with the clover Schur
    operator, so S_pf = |xi|^2 at the start (S_f - S_det, S_det from the library's
    log det); a short run accepts, and a trajectory is reversible."""
    lat = hr.Lattice((4, 4, 4, 4), 1)
    m0, csw = 0.1, 1.0
    q = dev(smeared(lat, 111))
    chain = HMC(ctx, lat, beta=2.2, m0=m0, fermions=True, n_steps=6, tau=0.5, seed=112, c_sw=csw)
    gen_state = chain.gen.get_state()
    eta = chain.draw_pseudofermion(q)
    chain.gen.set_state(gen_state)
    xi = chain._xi()
    clov = fields.build_clover(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_CLOVER_SW, m0, csw, q)
    S_det = -2.0 * hr.hr_clover_logdet(ctx, lat, hr.HR_FUND, clov, hr.HR_ODD)
    p = torch.zeros((4, int(np.prod(lat)), 3), dtype=torch.float64, device="cuda")
    prm = hr.hr_hmc_params_default(2.2, m0, True, 1, 1e-6)
    prm.clover, prm.c_sw = 1, csw
    prm.solver.tol = 1e-13
    info = hr.hr_hmc_trajectory(ctx, lat, prm, q.clone(), p, eta, chain.work)
    xi_h = fields.unpack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xi).cpu().numpy()
    want = float(np.vdot(xi_h, xi_h).real)
    assert abs(info.fermion_action_start - S_det - want) <= 1e-9 * want
    for _ in range(3):
        acc, info = chain.step(q)
        assert np.isfinite(info.dH) and abs(info.dH) < 2.0
    assert chain.accepted >= 2
    pp = torch.randn((4, int(np.prod(lat)), 3), dtype=torch.float64, device="cuda")
    q0 = q.clone()
    chain.prm.solver.tol = 1e-12
    i1 = hr.hr_hmc_trajectory(ctx, lat, chain.prm, q, pp, eta, chain.work)
    pp.neg_()
    i2 = hr.hr_hmc_trajectory(ctx, lat, chain.prm, q, pp, eta, chain.work)
    assert (q - q0).abs().max().item() <= 1e-9 and abs(i1.dH + i2.dH) <= 1e-7


@pytest.mark.parametrize("kind", [hr.HR_CLOVER_SW, hr.HR_CLOVER_EXP])
def test_clover_hasenbusch_trajectory_matches_oracle(ctx, kind):
    """Clover fermions with Hasenbusch's two pseudofermions (a heavy clover field
    beside the light one), on two time scales, against the oracle."""
    from oracle import clover as ocl

    lat = hr.Lattice((4, 2, 2, 4), 1)
    beta, m0, mh, csw = 2.2, 0.05, 0.5, 1.1
    q = smeared(lat, 121)
    p = np.random.default_rng(122).normal(size=(4, int(np.prod(lat)), 3))
    prm = hr.hr_hmc_params_default(beta, m0, True, 2, 0.3, hr.HR_INTEGRATOR_OMELYAN)
    prm.solver.tol = 1e-13
    prm.n_steps_gauge = 2
    prm.clover, prm.c_sw, prm.clover_kind = 1, csw, kind
    prm.hasenbusch, prm.m0_hasenbusch = 1, mh
    eta, eta_p = eta_field(ctx, lat, m0, 123)
    phi, phi_p = eta_field(ctx, lat, m0, 124)
    qg, pg, info = run_gpu(ctx, lat, q, p, prm, eta_p, phi_p)
    okind = ocl.KIND_EXP if kind == hr.HR_CLOVER_EXP else ocl.KIND_SW
    ferm = ocl.CloverHasenbusch(lat, m0, mh, csw, eta, phi, bc=1, kind=okind)
    qo, po, io = ohmc.trajectory(lat, q, p, beta, 2, 0.3, hr.HR_INTEGRATOR_OMELYAN, ferm, n_steps_gauge=2)
    assert np.abs(qg - qo).max() <= 1e-11
    assert np.abs(pg - po).max() <= 1e-9
    assert abs(info.dH - io["dH"]) <= 1e-9, (info.dH, io["dH"])
    assert abs(info.fermion_action_end - io["end"]["fermion"]) <= 1e-9 * abs(io["end"]["fermion"])


def test_clover_hasenbusch_chain(ctx):
    lat = hr.Lattice((4, 4, 4, 4), 1)
    q = dev(smeared(lat, 131))
    chain = HMC(ctx, lat, beta=2.2, m0=0.05, fermions=True, n_steps=4, tau=0.5, seed=132, c_sw=1.0,
                m0_hasenbusch=0.5, n_steps_gauge=2)
    for _ in range(3):
        acc, info = chain.step(q)
        assert np.isfinite(info.dH) and abs(info.dH) < 2.0
    assert chain.accepted >= 2
