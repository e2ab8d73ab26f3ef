"""The hop with a chunk of right-hand sides per thread (kernel variants 20 and
21: chunks of 2 and 4, FP32 and binary16 storage), forced through the tuning
cache, against the FP64 oracle and against the one-RHS-per-thread kernels.

Lattices with 360 and 144 sites per parity leave a ragged last 32-site block;
2, 4 and 32 right-hand sides put 16, 8 and 1 lattice sites in a block, so the
threads of a site, the chunk's right-hand sides r = t + k N / C and the
per-RHS reduction (shared-memory regrouping before the grid reduction) are
all exercised.  Tolerances: FP32 1e-6 against the oracle and against the
plain FP32 kernel (the same operations, other FMA contractions); binary16
4e-3 against the oracle and 2e-3 against the plain binary16 kernel (the
half2 projection rounds once more).  The mixed-precision solvers, whose
fused reductions run in these kernels, must reach the oracle's true
residual 1e-10 for every right-hand side.
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


def forced(tmp_path, monkeypatch, name, dims, prec, variant, block, n_rhs):
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


CASES = [((4, 6, 6, 10), 2), ((2, 4, 6, 6), 4), ((4, 6, 6, 10), 4), ((4, 6, 2, 6), 32)]


@pytest.mark.parametrize("prec", [hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("variant,block", [(20, 64), (20, 256), (21, 128), (21, 192), (21, 32)])
@pytest.mark.parametrize("dims,n_rhs", CASES, ids=[f"{d[0]}x{d[1]}x{d[2]}x{d[3]}_n{n}" for d, n in CASES])
def test_rhs_chunk_every_operator(tmp_path, monkeypatch, dims, n_rhs, variant, block, prec):
    q = synth.haar_links(dims, 83)
    psi = synth.gaussian_spinor(dims, 2, 84, n_rhs=n_rhs)
    base = forced(tmp_path, monkeypatch, "plain", dims, prec, 0, 128, n_rhs)
    chunk = forced(tmp_path, monkeypatch, "chunk", dims, prec, variant, block, n_rhs)
    assert hr.hr_tune_lookup(chunk, dims, hr.HR_FUND, prec, n_rhs) == (variant, block)
    L = oracle.expand_links(dims, 2, q)
    for (op, par, a), (_, _, b) in zip(apply_all(chunk, dims, prec, q, psi, n_rhs),
                                       apply_all(base, dims, prec, q, psi, n_rhs)):
        m = oracle.parity_mask(dims) == par
        assert rel(a[..., m, :, :], b[..., m, :, :]) <= AGREE[prec], (op, par)
        for r in sorted({0, n_rhs // 2 - 1, n_rhs // 2, n_rhs - 1}):
            want = oracle_op(dims, L, psi[r], op, par)
            tol = TOL[prec] * (3 if op == hr.HR_OP_NORMAL else 2 if op != hr.HR_OP_HOP else 1)
            assert rel(a[r][m], want[m]) <= tol, (op, par, r)
    base.close()
    chunk.close()


@pytest.mark.parametrize("prec", [hr.HR_F32, hr.HR_F16])
def test_rhs_chunk_antiperiodic(tmp_path, monkeypatch, prec):
    lat = hr.Lattice((4, 6, 6, 10), 15)
    c = forced(tmp_path, monkeypatch, "bc", lat, prec, 21, 64, 4)
    q = synth.haar_links(lat, 93)
    psi = synth.gaussian_spinor(lat, 2, 94, n_rhs=4)
    L = oracle.expand_links(lat, 2, q)
    for (op, par, got) in apply_all(c, lat, prec, q, psi, 4):
        m = oracle.parity_mask(lat) == par
        tol = TOL[prec] * (3 if op == hr.HR_OP_NORMAL else 2 if op != hr.HR_OP_HOP else 1)
        for r in (0, 3):
            assert rel(got[r][m], oracle_op(lat, L, psi[r], op, par, bc=15)[m]) <= tol, (op, par, r)
    c.close()


def test_rhs_chunk_one_rhs_runs_the_plain_kernel(tmp_path, monkeypatch):
    """A chunk variant forced for a single right-hand side has nothing to
    share: the dispatch runs the plain kernel, bit for bit."""
    dims = (4, 6, 6, 10)
    q = synth.haar_links(dims, 85)
    psi = synth.gaussian_spinor(dims, 2, 86)
    base = forced(tmp_path, monkeypatch, "plain1", dims, hr.HR_F32, 0, 128, 1)
    chunk = forced(tmp_path, monkeypatch, "chunk1", dims, hr.HR_F32, 20, 128, 1)
    for (_, _, a), (_, _, b) in zip(apply_all(chunk, dims, hr.HR_F32, q, psi, 1),
                                    apply_all(base, dims, hr.HR_F32, q, psi, 1)):
        assert np.array_equal(a, b)
    base.close()
    chunk.close()


@pytest.mark.parametrize("n_rhs,variant", [(2, 20), (4, 21), (32, 20), (32, 21)])
@pytest.mark.parametrize("inner", [hr.HR_F32, hr.HR_F16])
def test_rhs_chunk_inner_cg(tmp_path, monkeypatch, inner, n_rhs, variant):
    """Mixed-precision CG with the chunk kernel as its inner hop (its fused
    per-RHS reductions included): the oracle's true residual of every
    right-hand side <= 1e-10."""
    dims = (8, 8, 8, 8)
    c = forced(tmp_path, monkeypatch, "cg", dims, inner, variant, 128, n_rhs)
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, 1002), dims, 0.6)
    bs = synth.gaussian_spinor(dims, 2, 2022, n_rhs=n_rhs)
    odd = oracle.parity_mask(dims) == 1
    bs[:, odd] = 0
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    opts.reliable_delta = 0.01
    opts.n_rhs = n_rhs
    gauge = fields.pack_gauge(c, dims, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(bs))
    xp = fields.zeros_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, n_rhs)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(dims, hr.HR_FUND, opts))
    rc, info = hr.hr_cg_solve(c, dims, -0.2, hr.HR_FUND, opts, gauge, bp, xp, work)
    assert rc == hr.HR_OK
    xs = fields.unpack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp, n_rhs).cpu().numpy()
    L = oracle.expand_links(dims, 2, q)
    for r in range(n_rhs):
        res = np.linalg.norm(bs[r] - oracle.normal(dims, L, -0.2, xs[r])) / np.linalg.norm(bs[r])
        assert res <= 1e-10, (r, res)
    c.close()


@pytest.mark.parametrize("prec", [hr.HR_F32, hr.HR_F16])
def test_autotune_with_several_rhs_includes_the_chunks(tmp_path, monkeypatch, prec):
    """With 4 right-hand sides the tuner also times the chunk kernels; whatever
    it picks, the tuned hop matches the oracle for every right-hand side."""
    dims = (8, 8, 8, 8)
    n_rhs = 4
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    c = hr.Context(0)
    q = synth.haar_links(dims, 95)
    psi = synth.gaussian_spinor(dims, 2, 96, n_rhs=n_rhs)
    gauge = fields.pack_gauge(c, dims, hr.HR_FUND, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(c, dims, hr.HR_FUND, prec, hr.HR_ODD, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(dims, hr.HR_FUND, prec, hr.HR_EVEN, n_rhs)
    res = hr.hr_autotune_hop(c, dims, hr.HR_FUND, prec, hr.HR_EVEN, n_rhs, gauge, src, dst, reps=3)
    one = hr.hr_autotune_hop(c, dims, hr.HR_FUND, prec, hr.HR_EVEN, 1, gauge, src, dst, reps=3)
    # two more shapes (variants 20 and 21) at each of the four block sizes
    assert res.candidates >= one.candidates + 8 - 1
    assert hr.hr_tune_lookup(c, dims, hr.HR_FUND, prec, n_rhs) == (res.variant, res.block)
    hr.hr_dirac_eo(c, dims, 0.0, hr.HR_FUND, prec, hr.HR_EVEN, hr.HR_OP_HOP, n_rhs, gauge, src, dst)
    got = fields.unpack_spinor(c, dims, hr.HR_FUND, prec, hr.HR_EVEN, dst, n_rhs).cpu().numpy()
    L = oracle.expand_links(dims, 2, q)
    m = oracle.parity_mask(dims) == 0
    for r in range(n_rhs):
        want = -0.5 * oracle.hop(dims, L, psi[r], parity=0)
        assert rel(got[r][m], want[m]) <= TOL[prec], r
    c.close()
