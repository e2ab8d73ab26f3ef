"""The two-sites-per-thread hop (kernel variants 16 and 17: FP32 and binary16
storage, the two sites in the lanes of packed f32x2 FMAs), forced through the
tuning cache, against the FP64 oracle and against the one-site kernels.

Lattices with 360 and 144 sites per parity leave the last 64-site group
partly empty (the second lane repeats the first site and is not stored);
with 4 and 32 right-hand sides the two sites of a thread are different
lattice sites with their own links.  Tolerances: FP32 1e-6 against the
oracle and 1e-6 against the one-site FP32 kernel (the same operations, other
FMA contractions); binary16 4e-3 against the oracle and 2e-3 against the
one-site binary16 kernel.  Both mixed-precision solvers must still reach the
true residual 1e-10.
"""

import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

TOL = {hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}
AGREE = {hr.HR_F32: 1e-6, hr.HR_F16: 2e-3}


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def forced(tmp_path, monkeypatch, name, dims, prec, variant, block, n_rhs=1):
    key = f"hop:r0:p{prec}:{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}:n{n_rhs}"
    cache = tmp_path / f"{name}.json"
    cache.write_text(json.dumps({key: [variant, block]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    return hr.Context(0)


def apply_all(c, lat, prec, q, psi, n_rhs):
    gauge = fields.pack_gauge(c, lat, hr.HR_FUND, prec, fields.gauge_to_device(q))
    out = []
    for op, par in ((hr.HR_OP_HOP, hr.HR_EVEN), (hr.HR_OP_HOP, hr.HR_ODD), (hr.HR_OP_SCHUR, hr.HR_EVEN),
                    (hr.HR_OP_SCHUR_DAG, hr.HR_EVEN), (hr.HR_OP_NORMAL, hr.HR_EVEN)):
        src_par = (1 - par) if op == hr.HR_OP_HOP else hr.HR_EVEN
        src = fields.pack_spinor(c, lat, hr.HR_FUND, prec, src_par, fields.spinor_to_device(psi))
        dst = fields.empty_spinor(lat, hr.HR_FUND, prec, par, n_rhs)
        wb = hr.hr_dirac_workspace_bytes(lat, hr.HR_FUND, prec, op, n_rhs)
        work = fields.empty_bytes(wb) if wb else None
        hr.hr_dirac_eo(c, lat, -0.3, hr.HR_FUND, prec, par, op, n_rhs, gauge, src, dst, work)
        out.append((op, par, fields.unpack_spinor(c, lat, hr.HR_FUND, prec, par, dst, n_rhs).cpu().numpy()))
    return out


def oracle_op(lat, L, psi, op, par, bc=0):
    if op == hr.HR_OP_HOP:
        return -0.5 * oracle.hop(lat, L, psi, parity=par, bc=bc)
    pe = psi.copy()
    pe[oracle.parity_mask(lat) == 1] = 0
    if op == hr.HR_OP_NORMAL:
        return oracle.normal(lat, L, -0.3, pe, bc=bc)
    return oracle.schur(lat, L, -0.3, pe, dagger=op == hr.HR_OP_SCHUR_DAG, bc=bc)


CASES = [((4, 6, 6, 10), 1), ((2, 4, 6, 6), 1), ((4, 6, 6, 10), 4), ((4, 6, 2, 6), 32)]


@pytest.mark.parametrize("prec", [hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("variant,block", [(16, 64), (16, 256), (17, 128)])
@pytest.mark.parametrize("dims,n_rhs", CASES, ids=[f"{d[0]}x{d[1]}x{d[2]}x{d[3]}_n{n}" for d, n in CASES])
def test_pair_sites_every_operator(tmp_path, monkeypatch, dims, n_rhs, variant, block, prec):
    q = synth.haar_links(dims, 81)
    psi = synth.gaussian_spinor(dims, 2, 82, n_rhs=n_rhs) if n_rhs > 1 else synth.gaussian_spinor(dims, 2, 82)
    base = forced(tmp_path, monkeypatch, "plain", dims, prec, 0, 128, n_rhs)
    pair = forced(tmp_path, monkeypatch, "pair", dims, prec, variant, block, n_rhs)
    assert hr.hr_tune_lookup(pair, dims, hr.HR_FUND, prec, n_rhs) == (variant, block)
    L = oracle.expand_links(dims, 2, q)
    for (op, par, a), (_, _, b) in zip(apply_all(pair, dims, prec, q, psi, n_rhs),
                                       apply_all(base, dims, prec, q, psi, n_rhs)):
        m = oracle.parity_mask(dims) == par
        assert rel(a[..., m, :, :], b[..., m, :, :]) <= AGREE[prec], (op, par)
        for r in ((0, n_rhs - 1) if n_rhs > 1 else (None,)):
            got = a[r] if r is not None else a
            src = psi[r] if r is not None else psi
            want = oracle_op(dims, L, src, op, par)
            tol = TOL[prec] * (3 if op == hr.HR_OP_NORMAL else 2 if op != hr.HR_OP_HOP else 1)
            assert rel(got[m], want[m]) <= tol, (op, par, r)
    base.close()
    pair.close()


@pytest.mark.parametrize("prec", [hr.HR_F32, hr.HR_F16])
def test_pair_sites_antiperiodic(tmp_path, monkeypatch, prec):
    lat = hr.Lattice((4, 6, 6, 10), 15)
    c = forced(tmp_path, monkeypatch, "bc", lat, prec, 16, 128)
    q = synth.haar_links(lat, 91)
    psi = synth.gaussian_spinor(lat, 2, 92)
    L = oracle.expand_links(lat, 2, q)
    for (op, par, got) in apply_all(c, lat, prec, q, psi, 1):
        m = oracle.parity_mask(lat) == par
        tol = TOL[prec] * (3 if op == hr.HR_OP_NORMAL else 2 if op != hr.HR_OP_HOP else 1)
        assert rel(got[m], oracle_op(lat, L, psi, op, par, bc=15)[m]) <= tol, (op, par)
    c.close()


@pytest.mark.parametrize("n_rhs", [1, 4])
@pytest.mark.parametrize("inner", [hr.HR_F32, hr.HR_F16])
def test_pair_sites_inner_cg(tmp_path, monkeypatch, inner, n_rhs):
    """Mixed-precision CG with the two-site kernel as its inner hop: the
    oracle's true residual of every right-hand side <= 1e-10."""
    dims = (8, 8, 8, 8)
    c = forced(tmp_path, monkeypatch, "cg", dims, inner, 16, 128, n_rhs)
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, 1002), dims, 0.6)
    bs = synth.gaussian_spinor(dims, 2, 2012, n_rhs=n_rhs)
    odd = oracle.parity_mask(dims) == 1
    bs[:, odd] = 0
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    opts.reliable_delta = 0.01
    opts.n_rhs = n_rhs
    gauge = fields.pack_gauge(c, dims, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN,
                            fields.spinor_to_device(bs if n_rhs > 1 else bs[0]))
    xp = fields.zeros_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, n_rhs)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(dims, hr.HR_FUND, opts))
    rc, info = hr.hr_cg_solve(c, dims, -0.2, hr.HR_FUND, opts, gauge, bp, xp, work)
    assert rc == hr.HR_OK
    xs = fields.unpack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp, n_rhs).cpu().numpy()
    if n_rhs == 1:
        xs = xs[None]
    L = oracle.expand_links(dims, 2, q)
    for r in range(n_rhs):
        res = np.linalg.norm(bs[r] - oracle.normal(dims, L, -0.2, xs[r])) / np.linalg.norm(bs[r])
        assert res <= 1e-10, (r, res)
    c.close()
