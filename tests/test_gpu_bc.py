"""Antiperiodic fermion boundary conditions (``hr_lattice.bc``) on the GPU.

The library folds the boundary sign into the packed links of the last slice of
each antiperiodic direction; the oracle applies the factor -1 to the neighbour
value a hop fetches across the boundary (its definition, independent of that
trick).  Every operator, solver and link derivative is compared with the
oracle at the same tolerances as the periodic tests: FP64 1e-13, FP32 1e-6,
FP16 storage 4e-3 relative L2; solves to a true residual of 1e-10.

bc values: 1 (time), 9 (time and x3, the direction that stays inside a row of
the packed layout), 15 (all four).
"""

import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import autograd as ag  # noqa: E402
from paper_2411_18511_gb300 import fields, hr  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}
REPS = [hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT]
PRECS = [hr.HR_F64, hr.HR_F32, hr.HR_F16]


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


def hop_error(ctx, lat, rep, prec, q, psi):
    """Largest relative error of both parities' hops against the oracle."""
    nc = nc_of(rep)
    L = oracle.expand_links(lat, nc, q)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, fields.gauge_to_device(q))
    dpsi = fields.spinor_to_device(psi)
    worst = 0.0
    for out_par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(ctx, lat, rep, prec, 1 - out_par, dpsi)
        dst = fields.empty_spinor(lat, rep, prec, out_par)
        hr.hr_dirac_eo(ctx, lat, 0.1, rep, prec, out_par, hr.HR_OP_HOP, 1, gauge, src, dst)
        got = fields.unpack_spinor(ctx, lat, rep, prec, out_par, dst).cpu().numpy()
        m = oracle.parity_mask(lat) == out_par
        psi_in = psi.copy()
        psi_in[m] = 0
        want = -0.5 * oracle.hop(lat, L, psi_in, parity=out_par, bc=lat.bc)
        worst = max(worst, rel(got[m], want[m]))
    return worst


@pytest.mark.parametrize("bc", [1, 9, 15])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
@pytest.mark.parametrize("dims", [(6, 4, 2, 6), (4, 6, 8, 10)])
def test_hop_matches_oracle(ctx, dims, rep, prec, bc):
    lat = hr.Lattice(dims, bc)
    q = synth.haar_links(dims, 11)
    psi = synth.gaussian_spinor(dims, nc_of(rep), 12)
    assert hop_error(ctx, lat, rep, prec, q, psi) <= TOL[prec]
    # and the boundary made a difference
    L = oracle.expand_links(dims, nc_of(rep), q)
    assert rel(oracle.hop(dims, L, psi, bc=bc), oracle.hop(dims, L, psi)) > 1e-2


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rep", REPS)
def test_full_operator_matches_oracle(ctx, rep, prec):
    lat = hr.Lattice((4, 4, 4, 4), hr.HR_BC_ANTIPERIODIC(0))
    nc = nc_of(rep)
    q = synth.haar_links(lat, 21)
    psi = synth.gaussian_spinor(lat, nc, 22)
    gauge = fields.pack_gauge(ctx, lat, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, lat, rep, prec, hr.HR_FULL, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(lat, rep, prec, hr.HR_FULL)
    hr.hr_dirac_apply(ctx, lat, 0.1, rep, prec, gauge, src, dst)
    got = fields.unpack_spinor(ctx, lat, rep, prec, hr.HR_FULL, dst).cpu().numpy()
    want = oracle.dirac(lat, oracle.expand_links(lat, nc, q), 0.1, psi, bc=1)
    assert rel(got, want) <= TOL[prec]


@pytest.mark.parametrize("op", [hr.HR_OP_SCHUR, hr.HR_OP_SCHUR_DAG, hr.HR_OP_NORMAL])
@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
@pytest.mark.parametrize("rep", REPS)
def test_schur_operators_match_oracle(ctx, rep, prec, op):
    lat = hr.Lattice((4, 6, 8, 10), 9)
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
        want = oracle.normal(lat, L, m0, psi, bc=9)
    else:
        want = oracle.schur(lat, L, m0, psi, dagger=op == hr.HR_OP_SCHUR_DAG, bc=9)
    assert rel(got[even], want[even]) <= 10 * TOL[prec]


def _forced_context(tmp_path, monkeypatch, lat, rep, prec, variant, block):
    key = f"hop:r{rep}:p{prec}:{lat[0]}x{lat[1]}x{lat[2]}x{lat[3]}:n1"
    cache = tmp_path / f"bc_{rep}_{prec}_{variant}_{block}.json"
    cache.write_text(json.dumps({key: [variant, block]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    return hr.Context(0)


@pytest.mark.parametrize("variant", list(range(14)))
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_every_hop_variant_applies_the_boundary(tmp_path, monkeypatch, rep, variant):
    """Each kernel variant (the tuner's choices) with all four directions antiperiodic."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lat = hr.Lattice((4, 6, 8, 10), 15)
    c = _forced_context(tmp_path, monkeypatch, lat, rep, hr.HR_F64, variant, 128)
    v, _ = hr.hr_tune_lookup(c, lat, rep, hr.HR_F64)
    q = synth.haar_links(lat, 41)
    psi = synth.gaussian_spinor(lat, nc_of(rep), 42)
    assert hop_error(c, lat, rep, hr.HR_F64, q, psi) <= TOL[hr.HR_F64], (rep, variant, v)


def boundary_q0_zero_links(lat, seed):
    """Haar links whose boundary-slice links have q0 = 0 exactly (pure i a.s):
    the adjoint layout's boundary bit then sits on a signed zero."""
    q = synth.haar_links(lat, seed)
    x = np.indices(lat).reshape(4, -1).T
    for mu in range(4):
        sel = x[:, mu] == lat[mu] - 1
        v = q[mu, sel, 1:]
        q[mu, sel, 0] = 0.0
        q[mu, sel, 1:] = v / np.linalg.norm(v, axis=1, keepdims=True)
    return q


@pytest.mark.parametrize("prec", PRECS)
def test_adjoint_boundary_bit_on_a_zero_q0(ctx, prec):
    lat = hr.Lattice((4, 6, 2, 6), 15)
    q = boundary_q0_zero_links(lat, 51)
    psi = synth.gaussian_spinor(lat, 3, 52)
    assert hop_error(ctx, lat, hr.HR_ADJ, prec, q, psi) <= TOL[prec]


def run_cg(ctx, lat, rep, q, m0, b, inner, n_rhs=1):
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    opts.n_rhs = n_rhs
    gauge = fields.pack_gauge(ctx, lat, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(lat, rep, hr.HR_F64, hr.HR_EVEN, n_rhs)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(lat, rep, opts))
    rc, info = hr.hr_cg_solve(ctx, lat, m0, rep, opts, gauge, bp, xp, work)
    x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, xp, n_rhs).cpu().numpy()
    return rc, info, x


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_cg_true_residual(ctx, rep, inner):
    lat = hr.Lattice((8, 4, 6, 4), 1)
    m0 = -0.2
    nc = nc_of(rep)
    # zero-q0 boundary links: the mixed solvers' FP32/FP16 gauge copies must keep the adjoint bit
    q = boundary_q0_zero_links(lat, 61)
    b = synth.gaussian_spinor(lat, nc, 62)
    b[~even_mask(lat)] = 0
    rc, info, x = run_cg(ctx, lat, rep, q, m0, b, inner)
    assert rc == hr.HR_OK
    L = oracle.expand_links(lat, nc, q)
    res = np.linalg.norm(b - oracle.normal(lat, L, m0, x, bc=1)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert abs(res - info.true_rel_residual) <= 1e-11


def test_cg_multi_rhs(ctx):
    lat = hr.Lattice((6, 4, 4, 6), 9)
    m0 = -0.2
    n = 4
    q = synth.haar_links(lat, 71)
    bs = synth.gaussian_spinor(lat, 2, 72, n_rhs=n)
    bs[:, ~even_mask(lat)] = 0
    rc, info, xs = run_cg(ctx, lat, hr.HR_FUND, q, m0, bs, hr.HR_F32, n_rhs=n)
    assert rc == hr.HR_OK
    L = oracle.expand_links(lat, 2, q)
    for r in range(n):
        res = np.linalg.norm(bs[r] - oracle.normal(lat, L, m0, xs[r], bc=9)) / np.linalg.norm(bs[r])
        assert res <= 1e-10, (r, res)


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_batch_with_mixed_boundaries(ctx, rep):
    lats = [hr.Lattice((4, 4, 4, 4), 1), hr.Lattice((2, 4, 6, 8), 0), hr.Lattice((6, 4, 2, 6), 15)]
    m0 = -0.2
    nc = nc_of(rep)
    probs = []
    for k, lat in enumerate(lats):
        q = synth.haar_links(lat, 80 + k)
        b = synth.gaussian_spinor(lat, nc, 90 + k)
        b[~even_mask(lat)] = 0
        gauge = fields.pack_gauge(ctx, lat, rep, hr.HR_F64, fields.gauge_to_device(q))
        bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
        probs.append((q, b, gauge, bp, fields.zeros_spinor(lat, rep, hr.HR_F64, hr.HR_EVEN)))
    opts = hr.hr_solver_default_opts()
    work = fields.empty_bytes(hr.hr_cg_batch_workspace_bytes(lats, rep))
    rc, infos = hr.hr_cg_solve_batch(ctx, lats, m0, rep, opts, [p[2] for p in probs], [p[3] for p in probs],
                                     [p[4] for p in probs], work)
    assert rc == hr.HR_OK
    for k, lat in enumerate(lats):
        q, b, _, _, xp = probs[k]
        x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
        L = oracle.expand_links(lat, nc, q)
        res = np.linalg.norm(b - oracle.normal(lat, L, m0, x, bc=lat.bc)) / np.linalg.norm(b)
        assert res <= 1e-10, (lat, res)


@pytest.mark.parametrize("bc", [1, 10])
def test_force_and_link_grad(ctx, bc):
    lat = hr.Lattice((4, 6, 2, 6), bc)
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
    assert rel(F.cpu().numpy(), oracle.force(lat, L, a, b, bc=bc)) <= 1e-13
    G = torch.zeros((4, V, 4), dtype=torch.float64, device="cuda")
    hr.hr_link_grad(ctx, lat, ap, bp, 1.0, G)
    assert rel(G.cpu().numpy(), oracle.link_grad(lat, a, b, bc=bc)) <= 1e-13


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_full_lattice_solve(ctx, rep):
    lat = hr.Lattice((4, 4, 6, 4), 1)
    m0 = 0.05
    nc = nc_of(rep)
    q = synth.haar_links(lat, 111)
    b = synth.gaussian_spinor(lat, nc, 112)
    opts = hr.hr_solver_default_opts()
    opts.tol = 1e-11
    gauge = fields.pack_gauge(ctx, lat, rep, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(b))
    xp = fields.empty_spinor(lat, rep, hr.HR_F64, hr.HR_FULL)
    work = fields.empty_bytes(hr.hr_solve_full_workspace_bytes(lat, rep, opts, hr.HR_SYSTEM_D))
    rc, info = hr.hr_solve_full(ctx, lat, m0, rep, opts, hr.HR_SYSTEM_D, gauge, bp, xp, work)
    assert rc == hr.HR_OK
    x = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, hr.HR_FULL, xp).cpu().numpy()
    L = oracle.expand_links(lat, nc, q)
    res = np.linalg.norm(b - oracle.dirac(lat, L, m0, x, bc=1)) / np.linalg.norm(b)
    assert res <= 1e-9, res


def test_autograd_dirac_apply(ctx):
    lat = hr.Lattice((4, 6, 2, 6), 1)
    m0 = 0.1
    q = synth.haar_links(lat, 121)
    psi = synth.gaussian_spinor(lat, 2, 122)
    g = synth.gaussian_spinor(lat, 2, 123)
    qt = torch.tensor(q, device="cuda", requires_grad=True)
    pt = torch.tensor(psi, device="cuda", requires_grad=True)
    y = ag.DiracApply.apply(qt, pt, lat, m0)
    L = oracle.expand_links(lat, 2, q)
    assert rel(y.detach().cpu().numpy(), oracle.dirac(lat, L, m0, psi, bc=1)) <= 1e-13
    y.backward(torch.tensor(g, device="cuda"))
    want_psi = oracle.gamma5(oracle.dirac(lat, L, m0, oracle.gamma5(g), bc=1))
    assert rel(pt.grad.cpu().numpy(), want_psi) <= 1e-13
    assert rel(qt.grad.cpu().numpy(), -0.5 * oracle.link_grad(lat, g, psi, bc=1)) <= 1e-13


def test_boundary_bits_out_of_range(ctx):
    lat = hr.Lattice((4, 4, 4, 4), 16)
    q = fields.gauge_to_device(synth.haar_links((4, 4, 4, 4), 131))
    out = fields.empty_bytes(hr.hr_gauge_packed_bytes((4, 4, 4, 4), 0, 0))
    with pytest.raises(hr.HrError):
        hr.hr_gauge_pack(ctx, lat, hr.HR_FUND, hr.HR_F64, q, out)
