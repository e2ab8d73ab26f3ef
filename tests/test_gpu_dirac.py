"""Parity of the CUDA operators (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over the output field): FP64 1e-13, FP32 1e-6 (both
stated for the method), FP16 storage 4e-3 (binary16 has a unit roundoff of
2^-11 = 4.9e-4 on each stored spinor and link component; a hop sums 8 terms of
such inputs, so a few units of roundoff relative to the result's norm).
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}
REPS = [hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT]
PRECS = [hr.HR_F64, hr.HR_F32, hr.HR_F16]
# several 32-site blocks with a ragged tail, tiny lattices with extent 2, mixed extents
DIMS = [(2, 2, 2, 2), (6, 4, 2, 6), (4, 6, 8, 10), (8, 8, 8, 8)]


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


def setup_fields(dims, rep, seed):
    q = synth.haar_links(dims, seed)
    psi = synth.gaussian_spinor(dims, nc_of(rep), seed + 1)
    return q, psi


def parity_mask(dims, p):
    return oracle.parity_mask(dims) == p


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_spinor_pack_roundtrip(ctx, rep, prec):
    dims = (6, 4, 2, 6)
    _, psi = setup_fields(dims, rep, 5)
    d = fields.spinor_to_device(psi)
    for par in (hr.HR_EVEN, hr.HR_ODD, hr.HR_FULL):
        pk = fields.pack_spinor(ctx, dims, rep, prec, par, d)
        back = fields.unpack_spinor(ctx, dims, rep, prec, par, pk).cpu().numpy()
        mask = np.ones(len(psi), bool) if par == hr.HR_FULL else parity_mask(dims, par)
        # FP64 fields are stored as double-float pairs: 48 significant bits (2^-48 = 3.6e-15)
        tol = {hr.HR_F64: 4e-15, hr.HR_F32: 1e-7, hr.HR_F16: 1e-3}[prec]
        assert rel(back[mask], psi[mask]) <= tol
        assert np.all(back[~mask] == 0)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_hop_matches_oracle(ctx, rep, prec, dims):
    nc = nc_of(rep)
    q, psi = setup_fields(dims, rep, 11)
    L = oracle.expand_links(dims, nc, q)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    dpsi = fields.spinor_to_device(psi)
    for out_par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(ctx, dims, rep, prec, 1 - out_par, dpsi)
        dst = fields.empty_spinor(dims, rep, prec, out_par)
        hr.hr_dirac_eo(ctx, dims, 0.1, rep, prec, out_par, hr.HR_OP_HOP, 1, gauge, src, dst)
        got = fields.unpack_spinor(ctx, dims, rep, prec, out_par, dst).cpu().numpy()
        psi_in = psi.copy()
        psi_in[parity_mask(dims, out_par)] = 0
        want = -0.5 * oracle.hop(dims, L, psi_in, parity=out_par)
        m = parity_mask(dims, out_par)
        assert rel(got[m], want[m]) <= TOL[prec], (rep, prec, dims, out_par)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_full_operator_matches_oracle(ctx, rep, prec):
    dims = (4, 4, 4, 4)  # the 4^4 correctness configuration (m0 = 0.1)
    nc = nc_of(rep)
    q, psi = setup_fields(dims, rep, 21)
    L = oracle.expand_links(dims, nc, q)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_FULL, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_FULL)
    hr.hr_dirac_apply(ctx, dims, 0.1, rep, prec, gauge, src, dst)
    got = fields.unpack_spinor(ctx, dims, rep, prec, hr.HR_FULL, dst).cpu().numpy()
    assert rel(got, oracle.dirac(dims, L, 0.1, psi)) <= TOL[prec]


@pytest.mark.parametrize("op", [hr.HR_OP_SCHUR, hr.HR_OP_SCHUR_DAG, hr.HR_OP_NORMAL])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_schur_operators_match_oracle(ctx, rep, prec, op):
    dims = (4, 6, 8, 10)
    m0 = -0.2
    nc = nc_of(rep)
    q, psi = setup_fields(dims, rep, 31)
    even = parity_mask(dims, 0)
    psi[~even] = 0
    L = oracle.expand_links(dims, nc, q)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_EVEN, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(dims, rep, prec, op))
    hr.hr_dirac_eo(ctx, dims, m0, rep, prec, hr.HR_EVEN, op, 1, gauge, src, dst, work)
    got = fields.unpack_spinor(ctx, dims, rep, prec, hr.HR_EVEN, dst).cpu().numpy()
    if op == hr.HR_OP_SCHUR:
        want = oracle.schur(dims, L, m0, psi)
    elif op == hr.HR_OP_SCHUR_DAG:
        want = oracle.schur(dims, L, m0, psi, dagger=True)
    else:
        want = oracle.normal(dims, L, m0, psi)
    tol = TOL[prec] * (3 if op == hr.HR_OP_NORMAL else 2)
    assert rel(got[even], want[even]) <= tol


@pytest.mark.parametrize("n_rhs", [2, 4, 8, 32])
@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
def test_multi_rhs_hop_equals_single(ctx, n_rhs, prec):
    dims = (4, 6, 2, 6)
    rep = hr.HR_FUND
    q = synth.haar_links(dims, 41)
    psis = synth.gaussian_spinor(dims, 2, 42, n_rhs=n_rhs)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_ODD, fields.spinor_to_device(psis))
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN, n_rhs)
    hr.hr_dirac_eo(ctx, dims, 0.0, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, n_rhs, gauge, src, dst)
    got = fields.unpack_spinor(ctx, dims, rep, prec, hr.HR_EVEN, dst, n_rhs).cpu().numpy()
    for r in range(n_rhs):
        s1 = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_ODD, fields.spinor_to_device(psis[r]))
        d1 = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN)
        hr.hr_dirac_eo(ctx, dims, 0.0, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, 1, gauge, s1, d1)
        one = fields.unpack_spinor(ctx, dims, rep, prec, hr.HR_EVEN, d1).cpu().numpy()
        np.testing.assert_array_equal(got[r], one)


def test_invalid_arguments_return_codes(ctx):
    dims = (4, 4, 4, 4)
    g = fields.empty_bytes(hr.hr_gauge_packed_bytes(dims, 0, 0))
    s = fields.empty_spinor(dims, 0, 0, 0)
    o = fields.empty_spinor(dims, 0, 0, 0)
    L = hr.lib()
    lat = hr.lattice((4, 4, 4, 5))
    rc = L.hr_dirac_eo(ctx.handle, lat, 0.1, 0, 0, 0, hr.HR_OP_HOP, 1, hr._ptr(g), hr._ptr(s),
                       hr._ptr(o), None, 0, None)
    assert rc == hr.HR_ERR_UNSUPPORTED
    rc = L.hr_dirac_eo(ctx.handle, hr.lattice(dims), 0.1, 0, 0, 0, hr.HR_OP_HOP, 1, hr._ptr(g), None,
                       hr._ptr(o), None, 0, None)
    assert rc == hr.HR_ERR_INVALID_ARG
    rc = L.hr_dirac_eo(ctx.handle, hr.lattice(dims), 0.1, 0, 0, 0, hr.HR_OP_HOP, 3, hr._ptr(g), hr._ptr(s),
                       hr._ptr(o), None, 0, None)
    assert rc == hr.HR_ERR_UNSUPPORTED
    rc = L.hr_dirac_eo(ctx.handle, hr.lattice(dims), 0.1, 0, 0, 0, hr.HR_OP_SCHUR, 1, hr._ptr(g), hr._ptr(s),
                       hr._ptr(o), hr._ptr(g), 10, None)
    assert rc == hr.HR_ERR_WORKSPACE
    assert b"workspace" in L.hr_last_error(ctx.handle)
    rc = L.hr_dirac_eo(ctx.handle, hr.lattice(dims), 0.1, 7, 0, 0, hr.HR_OP_HOP, 1, hr._ptr(g), hr._ptr(s),
                       hr._ptr(o), None, 0, None)
    assert rc == hr.HR_ERR_INVALID_ARG
    # misaligned buffers are refused before any launch (the kernels move 16-byte vectors)
    big = fields.empty_bytes(hr.hr_spinor_packed_bytes(dims, 0, 0, 0, 1) + 64)
    for off in (4, 8):
        rc = L.hr_dirac_eo(ctx.handle, hr.lattice(dims), 0.1, 0, 0, 0, hr.HR_OP_HOP, 1, hr._ptr(g),
                           big.data_ptr() + off, hr._ptr(o), None, 0, None)
        assert rc == hr.HR_ERR_INVALID_ARG
        assert b"aligned" in L.hr_last_error(ctx.handle)
    rc = L.hr_gamma5(ctx.handle, hr.lattice(dims), 0, big.data_ptr() + 8, None)
    assert rc == hr.HR_ERR_INVALID_ARG
    res = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = L.hr_norm2_noalloc(hr.lattice(dims), 0, 1, big.data_ptr() + 4, res.data_ptr(), None)
    assert rc == hr.HR_ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_full_size_48_sampled_sites(ctx):
    """48^4 fundamental FP64 hop in the launch configuration the benchmark times,
    checked on 2000 sampled output sites against the oracle."""
    dims = (48, 48, 48, 48)
    rep, prec = hr.HR_FUND, hr.HR_F64
    q = synth.haar_links(dims, 1003)
    psi = synth.gaussian_spinor(dims, 2, 2003)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    dpsi = fields.spinor_to_device(psi)
    L = oracle.expand_links(dims, 2, q)
    rng = np.random.default_rng(7)
    for out_par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(ctx, dims, rep, prec, 1 - out_par, dpsi)
        dst = fields.empty_spinor(dims, rep, prec, out_par)
        hr.hr_dirac_eo(ctx, dims, 0.0, rep, prec, out_par, hr.HR_OP_HOP, 1, gauge, src, dst)
        got = fields.unpack_spinor(ctx, dims, rep, prec, out_par, dst).cpu().numpy()
        cand = np.where(parity_mask(dims, out_par))[0]
        sites = np.concatenate([cand[:16], cand[-16:], rng.choice(cand, 2000, replace=False)])
        psi_in = psi.copy()
        psi_in[parity_mask(dims, out_par)] = 0
        want = -0.5 * oracle.hop_sites(dims, L, psi_in, sites)
        assert rel(got[sites], want) <= 1e-13
    del L
