"""The binary16 hop with the spin projection in half2 arithmetic (kernel
variants 14, 15, their cp.async-staged forms 18, 19 and register-prefetch
forms 22, 23), forced through the tuning cache, against the FP64 oracle and
against the FP32-arithmetic binary16 kernel.

Tolerances: the stored binary16 components carry a relative rounding of 2^-11
of their site's largest component; the half2 projection adds one more such
rounding to each projected component, so the hop agrees with the oracle to
the FP16 tolerance of the other kernels (4e-3 relative L2) and with the plain
binary16 kernel to a few storage roundings (2e-3).  The FP16-inner CG must
still reach the true residual 1e-10, recomputed by the oracle.
"""

import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

DIMS = (4, 6, 6, 10)  # 360 sites per parity: a ragged last 32-site block


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def forced(tmp_path, monkeypatch, name, dims, variant, block, n_rhs=1, bc=0):
    key = f"hop:r0:p2:{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}:n{n_rhs}"
    cache = tmp_path / f"{name}.json"
    cache.write_text(json.dumps({key: [variant, block]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    return hr.Context(0)


def apply_all(c, lat, q, psi, n_rhs):
    """hop (both parities), Mhat, Mhat^+, Mhat^+ Mhat on binary16 fields."""
    prec = hr.HR_F16
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


def oracle_op(lat, L, psi, op, par):
    if op == hr.HR_OP_HOP:
        return -0.5 * oracle.hop(lat, L, psi, parity=par)
    pe = psi.copy()
    pe[oracle.parity_mask(lat) == 1] = 0
    if op == hr.HR_OP_NORMAL:
        return oracle.normal(lat, L, -0.3, pe)
    return oracle.schur(lat, L, -0.3, pe, dagger=op == hr.HR_OP_SCHUR_DAG)


@pytest.mark.parametrize("n_rhs", [1, 4])
@pytest.mark.parametrize("variant,block", [(14, 64), (14, 128), (15, 256), (18, 64), (18, 192), (19, 128),
                                           (22, 64), (23, 128)])
def test_half_variant_every_operator(tmp_path, monkeypatch, variant, block, n_rhs):
    q = synth.haar_links(DIMS, 61)
    psi = synth.gaussian_spinor(DIMS, 2, 62, n_rhs=n_rhs) if n_rhs > 1 else synth.gaussian_spinor(DIMS, 2, 62)
    base = forced(tmp_path, monkeypatch, "plain", DIMS, 0, 128, n_rhs)
    half = forced(tmp_path, monkeypatch, "half", DIMS, variant, block, n_rhs)
    assert hr.hr_tune_lookup(half, DIMS, hr.HR_FUND, hr.HR_F16, n_rhs) == (variant, block)
    L = oracle.expand_links(DIMS, 2, q)
    for (op, par, a), (_, _, b) in zip(apply_all(half, DIMS, q, psi, n_rhs), apply_all(base, DIMS, q, psi, n_rhs)):
        m = oracle.parity_mask(DIMS) == par
        assert rel(a[..., m, :, :], b[..., m, :, :]) <= 2e-3, (op, par)
        for r in range(n_rhs):
            got = a[r] if n_rhs > 1 else a
            src = psi[r] if n_rhs > 1 else psi
            want = oracle_op(DIMS, L, src, op, par)
            tol = 4e-3 * (3 if op == hr.HR_OP_NORMAL else 2 if op != hr.HR_OP_HOP else 1)
            assert rel(got[m], want[m]) <= tol, (op, par, r)
    base.close()
    half.close()


@pytest.mark.parametrize("variant", [14, 15, 18, 19, 22, 23])
def test_half_variant_antiperiodic(tmp_path, monkeypatch, variant):
    lat = hr.Lattice(DIMS, 15)
    c = forced(tmp_path, monkeypatch, "bc", lat, variant, 128)
    q = synth.haar_links(lat, 71)
    psi = synth.gaussian_spinor(lat, 2, 72)
    L = oracle.expand_links(lat, 2, q)
    gauge = fields.pack_gauge(c, lat, hr.HR_FUND, hr.HR_F16, fields.gauge_to_device(q))
    for par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(c, lat, hr.HR_FUND, hr.HR_F16, 1 - par, fields.spinor_to_device(psi))
        dst = fields.empty_spinor(lat, hr.HR_FUND, hr.HR_F16, par)
        hr.hr_dirac_eo(c, lat, 0.0, hr.HR_FUND, hr.HR_F16, par, hr.HR_OP_HOP, 1, gauge, src, dst)
        got = fields.unpack_spinor(c, lat, hr.HR_FUND, hr.HR_F16, par, dst).cpu().numpy()
        want = -0.5 * oracle.hop(lat, L, psi, parity=par, bc=15)
        m = oracle.parity_mask(lat) == par
        assert rel(got[m], want[m]) <= 4e-3
    c.close()


@pytest.mark.parametrize("variant", [14, 15, 18, 19, 22, 23])
def test_half_variant_inner_cg(tmp_path, monkeypatch, variant):
    """FP16-inner mixed-precision CG with the half2 kernel as its inner hop."""
    dims = (8, 8, 8, 8)
    c = forced(tmp_path, monkeypatch, "cg", dims, variant, 128)
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, 1002), dims, 0.6)
    b = synth.gaussian_spinor(dims, 2, 2002)
    b[oracle.parity_mask(dims) == 1] = 0
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = hr.HR_F16
    opts.reliable_delta = 0.01
    gauge = fields.pack_gauge(c, dims, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(dims, hr.HR_FUND, opts))
    rc, info = hr.hr_cg_solve(c, dims, -0.2, hr.HR_FUND, opts, gauge, bp, xp, work)
    assert rc == hr.HR_OK
    x = fields.unpack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
    L = oracle.expand_links(dims, 2, q)
    res = np.linalg.norm(b - oracle.normal(dims, L, -0.2, x)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    c.close()
