"""The clover term's HMC force and action on the GPU against the oracle
(oracle/clover.py: clover_derivative, CloverFermions, itself pinned by finite
differences of dense-matrix actions in tests/test_oracle_clover_force.py).
FP64 throughout: forces to 1e-12 relative L2, log det to 1e-12 relative."""

import numpy as np
import pytest

import oracle
import synth
from oracle import clover as ocl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import fields, hr  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def smeared(dims, seed):
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, seed), dims, 0.6)
    return q


@pytest.mark.parametrize("dims", [(4, 6, 2, 6), (2, 4, 4, 2)])
def test_insertion_force_matches_oracle(ctx, dims):
    V = int(np.prod(dims))
    q = synth.haar_links(dims, 601)
    rng = np.random.default_rng(602)
    lam = rng.normal(size=(V, 8, 8)) + 1j * rng.normal(size=(V, 8, 8))
    csw, coeff = 1.3, 0.7
    F = torch.zeros((4, V, 3), dtype=torch.float64, device="cuda")
    work = fields.empty_bytes(hr.hr_clover_force_workspace_bytes(dims))
    hr.hr_clover_insertion_force(ctx, dims, csw, fields.gauge_to_device(q), torch.tensor(lam, device="cuda"), coeff,
                                 F, work)
    want = coeff * csw * ocl.clover_derivative(dims, oracle.expand_links(dims, 2, q), lam)
    assert rel(F.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("kind", [hr.HR_CLOVER_SW, hr.HR_CLOVER_EXP])
@pytest.mark.parametrize("with_det", [0, 1])
@pytest.mark.parametrize("lat", [hr.Lattice((4, 6, 2, 6)), hr.Lattice((4, 4, 4, 4), 1),
                                 hr.Lattice((4, 2, 4, 6), 1, (0.4, 0.0, -1.2, 0.9))])
def test_fermion_force_matches_oracle(ctx, lat, with_det, kind):
    m0, csw = 0.1, 1.2
    V = int(np.prod(lat))
    q = smeared(lat, 611)
    X = synth.gaussian_spinor(lat, 2, 612)
    X[oracle.parity_mask(lat) == 1] = 0
    qd = fields.gauge_to_device(q)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, qd)
    clov = fields.build_clover(ctx, lat, hr.HR_FUND, hr.HR_F64, kind, m0, csw, qd)
    Xp = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(X))
    F = torch.zeros((4, V, 3), dtype=torch.float64, device="cuda")
    work = fields.empty_bytes(hr.hr_clover_force_workspace_bytes(lat))
    hr.hr_clover_fermion_force(ctx, lat, m0, csw, qd, gauge, clov, Xp, with_det, 0.5, F, work, kind=kind)
    ferm = ocl.CloverFermions(lat, m0, csw, np.zeros_like(X), bc=lat.bc,
                              kind=ocl.KIND_EXP if kind == hr.HR_CLOVER_EXP else ocl.KIND_SW)
    want = 0.5 * ferm.force_at(q, X, det=bool(with_det))
    assert rel(F.cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_logdet_matches_oracle(ctx, rep):
    lat = (4, 6, 2, 6)
    nc = 2 if rep == hr.HR_FUND else 3
    m0, csw = 0.1, 1.2
    q = smeared(lat, 621)
    A = ocl.site_term(lat, oracle.expand_links(lat, nc, q), m0, csw, ocl.KIND_SW)
    clov = fields.build_clover(ctx, lat, rep, hr.HR_F64, hr.HR_CLOVER_SW, m0, csw, fields.gauge_to_device(q))
    for par in (hr.HR_EVEN, hr.HR_ODD):
        m = oracle.parity_mask(lat) == par
        want = float(np.sum(np.linalg.slogdet(A[m])[1]))
        got = hr.hr_clover_logdet(ctx, lat, rep, clov, par)
        assert abs(got - want) <= 1e-12 * abs(want), (par, got, want)


def test_argument_checks(ctx):
    lat = hr.Lattice((4, 4, 4, 4))
    V = int(np.prod(lat))
    q = synth.haar_links(lat, 631)
    qd = fields.gauge_to_device(q)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, qd)
    clov = fields.build_clover(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_CLOVER_SW, 0.1, 1.0, qd)
    X = fields.zeros_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    F = torch.zeros((4, V, 3), dtype=torch.float64, device="cuda")
    need = hr.hr_clover_force_workspace_bytes(lat)
    L = hr.lib()
    small = fields.empty_bytes(need - 256)
    rc = L.hr_clover_fermion_force(ctx.handle, hr.lattice(lat), 0, 0.1, 1.0, hr._ptr(qd), hr._ptr(gauge),
                                   hr._ptr(clov), hr._ptr(X), None, 1, 1.0, hr._ptr(F), hr._ptr(small), need - 256, None)
    assert rc == hr.HR_ERR_WORKSPACE
    work = fields.empty_bytes(need)
    rc = L.hr_clover_fermion_force(ctx.handle, hr.lattice(lat), 7, 0.1, 1.0, hr._ptr(qd), hr._ptr(gauge),
                                   hr._ptr(clov), hr._ptr(X), None, 1, 1.0, hr._ptr(F), hr._ptr(work), need, None)
    assert rc == hr.HR_ERR_INVALID_ARG
    big = fields.empty_bytes(hr.hr_spinor_packed_bytes(lat, 0, 0, 0, 1) + 64)
    rc = L.hr_clover_fermion_force(ctx.handle, hr.lattice(lat), 0, 0.1, 1.0, hr._ptr(qd), hr._ptr(gauge),
                                   hr._ptr(clov), big.data_ptr() + 8, None, 1, 1.0, hr._ptr(F), hr._ptr(work), need, None)
    assert rc == hr.HR_ERR_INVALID_ARG
    # a site block that is not positive definite: log det refuses it
    rough = fields.build_clover(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_CLOVER_SW, 0.1, 60.0, qd)
    with pytest.raises(hr.HrError, match="positive definite"):
        hr.hr_clover_logdet(ctx, lat, hr.HR_FUND, rough, hr.HR_ODD)
    # a clover kind the trajectory driver does not know
    prm = hr.hr_hmc_params_default(2.2, 0.1, True, 2, 0.2)
    prm.clover, prm.c_sw, prm.clover_kind = 1, 1.0, 5
    work_h = fields.empty_bytes(hr.hr_hmc_workspace_bytes(lat, prm))
    p = torch.zeros((4, V, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(hr.HrError) as err:
        hr.hr_hmc_trajectory(ctx, lat, prm, qd.clone(), p, X, work_h)
    assert err.value.code == hr.HR_ERR_INVALID_ARG
