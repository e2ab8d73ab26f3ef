"""The pseudofermion force entry points through the C ABI, against the oracle.

hr_fermion_force / hr_fermion_link_grad give coeff * d/d(links) Re<L, Mhat^+
Mhat X> at fixed even fields X, L.  With c = 1/(4(4+m0)) and H_eo^+ = g5 H_oe g5
the oracle's form of that derivative is

    -c [ dRe<(Mhat L, H_eo^+ Mhat L), H (X, H_oe X)> + dRe<(Mhat X, ...), H (L, H_oe L)> ]

with every piece (Schur operator, hops, the hop derivative) taken from the
oracle, whose force is pinned by finite differences in the oracle tests.  For
the HMC's S = Re<eta, (Mhat^+ Mhat)^-1 eta>: L = X = the oracle's solution,
coeff = -1.  hr_dot is checked against numpy.
"""

import ctypes

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


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def oracle_pair(lat, L, m0, Y_src, Z, **kw):
    """Full fields a = (Mhat Y, H_eo^+ Mhat Y) and b = (Z, H_oe Z) by the oracle."""
    even = oracle.parity_mask(lat) == 0
    Y = oracle.schur(lat, L, m0, Y_src, **kw)
    W = oracle.gamma5(oracle.hop(lat, L, oracle.gamma5(Y), parity=1, **kw))
    HZ = oracle.hop(lat, L, Z, parity=1, **kw)
    a = np.where(even[:, None, None], Y, W)
    b = np.where(even[:, None, None], Z, HZ)
    return a, b


def oracle_deriv(lat, L, m0, X, Lam, grad, **kw):
    c = 1.0 / (4.0 * (4.0 + m0))
    f = (lambda a, b: oracle.link_grad(lat, a, b, **kw)) if grad else (lambda a, b: oracle.force(lat, L, a, b, **kw))
    t1 = f(*oracle_pair(lat, L, m0, Lam, X, **kw))
    t2 = f(*oracle_pair(lat, L, m0, X, Lam, **kw))
    return -c * (t1 + t2)


LATS = [hr.Lattice((4, 4, 4, 4)), hr.Lattice((4, 6, 2, 6), 1), hr.Lattice((6, 4, 4, 2), 9, (0.4, 0.0, -1.1, 0.0))]


@pytest.mark.parametrize("grad", [False, True])
@pytest.mark.parametrize("lat", LATS, ids=["periodic", "antiperiodic_t", "twisted"])
def test_fermion_deriv_matches_oracle(ctx, lat, grad):
    m0 = -0.2
    kw = {"bc": lat.bc, "theta": lat.theta}
    q = synth.haar_links(lat, 301)
    X = synth.gaussian_spinor(lat, 2, 302)
    Lam = synth.gaussian_spinor(lat, 2, 303)
    odd = oracle.parity_mask(lat) == 1
    X[odd] = 0
    Lam[odd] = 0
    L = oracle.expand_links(lat, 2, q)
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    Xp = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(X))
    Lp = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(Lam))
    V = int(np.prod(lat))
    out = torch.zeros((4, V, 4 if grad else 3), dtype=torch.float64, device="cuda")
    work = fields.empty_bytes(hr.hr_fermion_force_workspace_bytes(lat))
    fn = hr.lib().hr_fermion_link_grad if grad else hr.lib().hr_fermion_force
    s = torch.cuda.current_stream().cuda_stream
    # through the C ABI: the symmetric form (L = NULL) and two distinct fields
    rc = fn(ctx.handle, hr.lattice(lat), m0, hr.HR_FUND, gauge.data_ptr(), Xp.data_ptr(), None, 0.5, out.data_ptr(),
            work.data_ptr(), work.numel(), s)
    assert rc == hr.HR_OK
    got = out.cpu().numpy()
    want = 0.5 * oracle_deriv(lat, L, m0, X, X, grad, **kw)
    assert rel(got, want) <= 1e-12
    out.zero_()
    rc = fn(ctx.handle, hr.lattice(lat), m0, hr.HR_FUND, gauge.data_ptr(), Xp.data_ptr(), Lp.data_ptr(), -1.0,
            out.data_ptr(), work.data_ptr(), work.numel(), s)
    assert rc == hr.HR_OK
    assert rel(out.cpu().numpy(), -oracle_deriv(lat, L, m0, X, Lam, grad, **kw)) <= 1e-12


def test_hmc_force_of_the_solution_matches_oracle(ctx):
    """S = Re<eta, (Mhat^+ Mhat)^-1 eta>: X from the library's CG, force with
    L = NULL and coeff = -1, against 2c dRe<(Y, W), H (X, Z)> of the oracle's
    own solve; the action through hr_dot against numpy."""
    lat = hr.Lattice((4, 4, 4, 8), 1)
    m0 = 0.1
    q = synth.haar_links(lat, 311)
    eta = synth.gaussian_spinor(lat, 2, 312)
    even = oracle.parity_mask(lat) == 0
    eta[~even] = 0
    L = oracle.expand_links(lat, 2, q)
    Xo, it, tr, ok = oracle.cg(lat, L, m0, eta, tol=1e-14, maxiter=5000, bc=1)
    assert ok
    gauge = fields.pack_gauge(ctx, lat, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    ep = fields.pack_spinor(ctx, lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(eta))
    opts = hr.hr_solver_default_opts()
    opts.tol = 1e-13
    xp = fields.zeros_spinor(lat, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    rc, _ = hr.hr_cg_solve(ctx, lat, m0, hr.HR_FUND, opts, gauge, ep, xp,
                           fields.empty_bytes(hr.hr_cg_workspace_bytes(lat, hr.HR_FUND, opts)))
    assert rc == hr.HR_OK
    F = torch.zeros((4, int(np.prod(lat)), 3), dtype=torch.float64, device="cuda")
    hr.hr_fermion_force(ctx, lat, m0, hr.HR_FUND, gauge, xp, None, -1.0, F,
                        fields.empty_bytes(hr.hr_fermion_force_workspace_bytes(lat)))
    c = 1.0 / (4 * (4 + m0))
    want = 2 * c * oracle.force(lat, L, *oracle_pair(lat, L, m0, Xo, Xo, bc=1), bc=1)
    assert rel(F.cpu().numpy(), want) <= 1e-10
    S = hr.hr_dot(ctx, lat, hr.HR_FUND, ep, xp)
    S_np = np.vdot(eta[even], Xo[even])
    assert abs(S.real - S_np.real) <= 1e-11 * abs(S_np.real)
    assert abs(S.imag) <= 1e-10 * abs(S_np.real)  # <eta, A^-1 eta> is real


def test_dot_matches_numpy(ctx):
    lat = (4, 6, 6, 10)
    a = synth.gaussian_spinor(lat, 3, 321)
    b = synth.gaussian_spinor(lat, 3, 322)
    odd = oracle.parity_mask(lat) == 1
    for rep in (hr.HR_ADJ, hr.HR_ADJ_MAT):
        ap = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_ODD, fields.spinor_to_device(a))
        bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_ODD, fields.spinor_to_device(b))
        got = hr.hr_dot(ctx, lat, rep, ap, bp)
        want = np.vdot(a[odd], b[odd])
        assert abs(got - want) <= 1e-13 * np.linalg.norm(a[odd]) * np.linalg.norm(b[odd])


def test_fermion_force_rejects_bad_arguments(ctx):
    lat = (4, 4, 4, 4)
    gauge = fields.empty_bytes(hr.hr_gauge_packed_bytes(lat, 0, 0))
    X = fields.zeros_spinor(lat, 0, 0, hr.HR_EVEN)
    F = torch.zeros((4, 256, 3), dtype=torch.float64, device="cuda")
    need = hr.hr_fermion_force_workspace_bytes(lat)
    assert need == 5 * hr.hr_spinor_packed_bytes(lat, 0, 0, hr.HR_EVEN, 1)
    work = fields.empty_bytes(need)
    Lb = hr.lib()
    s = torch.cuda.current_stream().cuda_stream
    args = lambda rep, x, wb: (ctx.handle, hr.lattice(lat), -0.2, rep, gauge.data_ptr(), x, None, 1.0,  # noqa: E731
                               F.data_ptr(), work.data_ptr(), wb, s)
    assert Lb.hr_fermion_force(*args(hr.HR_ADJ, X.data_ptr(), need)) == hr.HR_ERR_UNSUPPORTED
    assert Lb.hr_fermion_force(*args(hr.HR_FUND, X.data_ptr(), need - 16)) == hr.HR_ERR_WORKSPACE
    assert Lb.hr_fermion_force(*args(hr.HR_FUND, None, need)) == hr.HR_ERR_INVALID_ARG
    assert Lb.hr_fermion_link_grad(*args(7, X.data_ptr(), need)) == hr.HR_ERR_INVALID_ARG
    re, im = ctypes.c_double(), ctypes.c_double()
    assert Lb.hr_dot(ctx.handle, hr.lattice(lat), 0, X.data_ptr(), None, ctypes.byref(re), ctypes.byref(im),
                     s) == hr.HR_ERR_INVALID_ARG
    assert hr.hr_fermion_force_workspace_bytes((4, 4, 4, 5)) == 0
