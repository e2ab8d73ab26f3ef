"""The hop autotuner and its kernel variants (registers-only, cp.async staged,
looped, bulk-copy tiled, ...), checked against the oracle for every shape the
tuner may choose."""

import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def hop_error(ctx, dims, rep, prec, seed=5):
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, seed)
    psi = synth.gaussian_spinor(dims, nc, seed + 1)
    L = oracle.expand_links(dims, nc, q)
    gauge = fields.pack_gauge(ctx, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(ctx, dims, rep, prec, hr.HR_ODD, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN)
    hr.hr_dirac_eo(ctx, dims, 0.0, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, 1, gauge, src, dst)
    got = fields.unpack_spinor(ctx, dims, rep, prec, hr.HR_EVEN, dst).cpu().numpy()
    even = oracle.parity_mask(dims) == 0
    pin = psi.copy()
    pin[even] = 0
    want = -0.5 * oracle.hop(dims, L, pin, parity=0)
    return np.linalg.norm(got[even] - want[even]) / np.linalg.norm(want[even])


def key(dims, rep, prec, n_rhs=1):
    return f"hop:r{rep}:p{prec}:{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}:n{n_rhs}"


@pytest.mark.parametrize("variant,block", [(0, 64), (0, 256), (1, 64), (1, 192), (2, 128), (2, 256), (3, 64), (3, 128), (4, 128), (4, 256), (5, 64), (5, 128), (6, 128), (6, 256), (7, 64), (7, 128), (7, 256),
                                           (8, 64), (8, 128), (8, 256), (9, 64), (9, 128), (10, 64),
                                           (10, 256), (11, 64), (11, 256), (12, 128), (13, 128), (14, 64),
                                           (14, 256), (15, 128), (15, 256), (16, 64), (16, 256), (17, 128), (18, 64),
                                           (18, 256), (19, 128), (22, 64), (23, 256)])
def test_forced_shapes_from_cache_match_oracle(tmp_path, monkeypatch, variant, block):
    dims = (6, 4, 2, 6)  # 144 sites per parity: ragged last block of 32
    cache = tmp_path / "tune.json"
    entries = {}
    for rep in (hr.HR_FUND, hr.HR_ADJ):
        for prec in (hr.HR_F64, hr.HR_F32, hr.HR_F16):
            entries[key(dims, rep, prec)] = [variant, block]
    cache.write_text(json.dumps(entries))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    c = hr.Context(0)
    for rep in (hr.HR_FUND, hr.HR_ADJ):
        for prec in (hr.HR_F64, hr.HR_F32, hr.HR_F16):
            assert hr.hr_tune_lookup(c, dims, rep, prec) == (variant, block)
            assert hop_error(c, dims, rep, prec) <= TOL[prec], (rep, prec, variant, block)
    c.close()


@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_autotune_chooses_and_persists(tmp_path, monkeypatch, rep, prec):
    dims = (8, 8, 8, 8)
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    c = hr.Context(0)
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, 9)
    psi = synth.gaussian_spinor(dims, nc, 10)
    gauge = fields.pack_gauge(c, dims, rep, prec, fields.gauge_to_device(q))
    src = fields.pack_spinor(c, dims, rep, prec, hr.HR_ODD, fields.spinor_to_device(psi))
    dst = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN)
    res = hr.hr_autotune_hop(c, dims, rep, prec, hr.HR_EVEN, 1, gauge, src, dst, reps=5)
    assert res.variant in range(24) and res.block in (64, 128, 192, 256)
    # the winner is the best median of four timings of the fastest shapes
    assert res.candidates >= 4 and 0 < res.best_ms <= 1.1 * res.default_ms
    assert hr.hr_tune_lookup(c, dims, rep, prec) == (res.variant, res.block)
    saved = json.loads(cache.read_text())
    assert saved[key(dims, rep, prec)] == [res.variant, res.block]
    # the reducing form (aux read, |out|^2 over the grid) keeps a choice of its own
    fin = saved[key(dims, rep, prec) + ":fin"]
    assert fin[0] in range(24) and fin[1] in (64, 128, 192, 256)
    assert res.candidates >= 8
    assert hop_error(c, dims, rep, prec) <= TOL[prec]
    c.close()
    c2 = hr.Context(0)
    assert hr.hr_tune_lookup(c2, dims, rep, prec) == (res.variant, res.block)
    c2.close()


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
def test_reducing_shape_from_cache_drives_the_solver(tmp_path, monkeypatch, inner):
    """A ':fin' cache entry sets the shape of the reducing launches only (the
    Schur operator's second hop and the CG's fused update), apart from the
    plain hops' shape; the solve stays right: the oracle recomputes its true
    residual, and x equals the one solved with the plain shape everywhere to
    the solver's tolerance."""
    dims = (6, 4, 8, 10)
    m0 = -0.2
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, 1002), dims, 0.6)
    b = synth.gaussian_spinor(dims, 2, 2006)
    b[oracle.parity_mask(dims) == 1] = 0
    red = {hr.HR_F64: [12, 192], hr.HR_F32: [7, 128], hr.HR_F16: [23, 128]}[inner]
    xs = []
    for with_fin in (False, True):
        entries = {}
        for p, sh in ((hr.HR_F64, [0, 64]), (inner, [0, 64])):
            entries[key(dims, hr.HR_FUND, p)] = sh
        if with_fin:
            entries[key(dims, hr.HR_FUND, inner) + ":fin"] = red
        cache = tmp_path / f"fin{int(with_fin)}.json"
        cache.write_text(json.dumps(entries))
        monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
        c = hr.Context(0)
        opts = hr.hr_solver_default_opts()
        opts.inner_prec = inner
        opts.reliable_delta = 0.1 if inner == hr.HR_F64 else (1e-5 if inner == hr.HR_F32 else 3e-3)
        gauge = fields.pack_gauge(c, dims, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
        bp = fields.pack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
        xp = fields.zeros_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
        work = fields.empty_bytes(hr.hr_cg_workspace_bytes(dims, hr.HR_FUND, opts))
        rc, info = hr.hr_cg_solve(c, dims, m0, hr.HR_FUND, opts, gauge, bp, xp, work)
        assert rc == hr.HR_OK
        assert hr.hr_tune_lookup(c, dims, hr.HR_FUND, inner) == (0, 64)
        x = fields.unpack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
        L = oracle.expand_links(dims, 2, q)
        r = b - oracle.normal(dims, L, m0, x)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
        xs.append(x)
        c.close()
    even = oracle.parity_mask(dims) == 0
    # both stop at a true residual of 1e-10: x agrees to about cond(A) x 1e-10
    assert np.linalg.norm((xs[0] - xs[1])[even]) / np.linalg.norm(xs[0][even]) < 1e-6


def test_autotune_rejects_bad_arguments(ctx):
    dims = (4, 4, 4, 4)
    g = fields.empty_bytes(hr.hr_gauge_packed_bytes(dims, 0, 0))
    s = fields.empty_spinor(dims, 0, 0, 0)
    with pytest.raises(hr.HrError):
        hr.hr_autotune_hop(ctx, dims, 0, 0, hr.HR_FULL, 1, g, s, fields.empty_spinor(dims, 0, 0, 0))
    with pytest.raises(hr.HrError):
        hr.hr_autotune_hop(ctx, dims, 0, 0, hr.HR_EVEN, 1, g, s, s)
    with pytest.raises(hr.HrError):
        hr.hr_autotune_hop(ctx, dims, 0, 0, hr.HR_EVEN, 1, g, s, fields.empty_spinor(dims, 0, 0, 0), reps=0)


def _forced_context(tmp_path, monkeypatch, name, dims, reps, precs, n_rhs, variant, block):
    cache = tmp_path / f"{name}.json"
    cache.write_text(json.dumps({key(dims, r, p, n_rhs): [variant, block] for r in reps for p in precs}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    return hr.Context(0)


@pytest.mark.parametrize("n_rhs", [1, 4])
@pytest.mark.parametrize("variant,block", [(8, 64), (8, 256), (9, 128), (10, 128), (10, 192), (11, 128),
                                           (11, 192), (12, 64), (13, 128)])
def test_variant_bitwise_equals_plain(tmp_path, monkeypatch, variant, block, n_rhs):
    """The bulk-copy tiled kernels (8, 9) take the near-direction neighbours
    from shared memory, the paired kernels (10-13) run two colours (adjoint:
    re and im) per f32x2 instruction and rebuild the adjoint links two entries
    at a time; in double-float all form every sum
    in the plain kernel's order, so every operator (hop, Schur, normal: g5
    inputs, aux terms, fused norms) must agree bit for bit (FP32 paired: to
    rounding), on a lattice whose tiles straddle rows, wraps and a ragged end,
    for quaternion and stored-matrix adjoint links."""
    dims = (4, 6, 6, 10)  # h3 = 5, 360 sites per parity
    reps, precs = (hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT), (hr.HR_F64, hr.HR_F32)
    base = _forced_context(tmp_path, monkeypatch, "plain", dims, reps, precs, n_rhs, 0, 128)
    tiled = _forced_context(tmp_path, monkeypatch, "tiled", dims, reps, precs, n_rhs, variant, block)
    for rep in reps:
        nc = 2 if rep == hr.HR_FUND else 3
        q = synth.haar_links(dims, 31)
        psi = synth.gaussian_spinor(dims, nc, 32, n_rhs=n_rhs) if n_rhs > 1 else synth.gaussian_spinor(dims, nc, 32)
        for prec in precs:
            assert hr.hr_tune_lookup(tiled, dims, rep, prec, n_rhs) == (variant, block)
            outs = []
            for c in (base, tiled):
                gauge = fields.pack_gauge(c, dims, rep, prec, fields.gauge_to_device(q))
                res = []
                for op, par in ((hr.HR_OP_HOP, hr.HR_EVEN), (hr.HR_OP_HOP, hr.HR_ODD),
                                (hr.HR_OP_SCHUR, hr.HR_EVEN), (hr.HR_OP_SCHUR_DAG, hr.HR_EVEN),
                                (hr.HR_OP_NORMAL, hr.HR_EVEN)):
                    src_par = (1 - par) if op == hr.HR_OP_HOP else hr.HR_EVEN
                    src = fields.pack_spinor(c, dims, rep, prec, src_par, fields.spinor_to_device(psi))
                    dst = fields.empty_spinor(dims, rep, prec, par, n_rhs)
                    wb = hr.hr_dirac_workspace_bytes(dims, rep, prec, op, n_rhs)
                    work = fields.empty_bytes(wb) if wb else None
                    hr.hr_dirac_eo(c, dims, -0.3, rep, prec, par, op, n_rhs, gauge, src, dst, work)
                    res.append(fields.unpack_spinor(c, dims, rep, prec, par, dst, n_rhs).cpu().numpy())
                outs.append(res)
            for a, b in zip(*outs):
                if prec == hr.HR_F32 and variant in (10, 11) and rep == hr.HR_FUND:
                    # FP32 arithmetic: the compiler contracts the plain kernel's
                    # products into FMAs its own way; agreement to rounding
                    assert np.linalg.norm(a - b) <= 2e-7 * np.linalg.norm(b), (rep, prec)
                else:
                    assert np.array_equal(a, b), (rep, prec)
    base.close()
    tiled.close()


def _spinor_padding_bytes(dims, rep, prec, n_rhs=1):
    """Byte offsets of the padding lanes (virtual sites >= V_h N) of one packed
    spinor half: the ragged last 32-site block, and the FP16 scales after it."""
    nc = 2 if rep == hr.HR_FUND else 3
    vh = int(np.prod(dims)) // 2
    nv = vh * n_rhs
    nblk = (nv + 31) // 32
    nvec = {hr.HR_F64: 4 * nc, hr.HR_F32: 2 * nc, hr.HR_F16: nc}[prec]
    idx = []
    for j in range(nv, nblk * 32):
        for v in range(nvec):
            base = (((j // 32) * nvec + v) * 32 + (j % 32)) * 16
            idx.extend(range(base, base + 16))
        if prec == hr.HR_F16:
            base = nblk * 32 * nvec * 16 + 4 * j
            idx.extend(range(base, base + 4))
    return np.asarray(idx, dtype=np.int64)


def _gauge_padding_bytes(dims, prec):
    """Byte offsets of the padding lanes (sites >= V_h) of a packed quaternion gauge."""
    vh = int(np.prod(dims)) // 2
    nblk = (vh + 31) // 32
    per = {hr.HR_F64: 16, hr.HR_F32: 16, hr.HR_F16: 8}[prec]
    nv = 2 if prec == hr.HR_F64 else 1
    idx = []
    for slot in range(8 * nblk):
        if slot % nblk != nblk - 1:
            continue
        for lane in range(vh - (nblk - 1) * 32, 32):
            for v in range(nv):
                base = ((slot * nv + v) * 32 + lane) * per
                idx.extend(range(base, base + per))
    return np.asarray(idx, dtype=np.int64)


@pytest.mark.parametrize("variant,block", [(0, 64), (1, 128), (2, 64), (4, 128), (6, 128), (7, 64), (8, 64),
                                           (10, 64), (11, 128), (14, 64), (15, 128), (16, 64), (17, 128), (18, 64),
                                           (19, 128), (22, 64), (23, 128)])
def test_padding_lanes_are_never_read(tmp_path, monkeypatch, variant, block):
    """NaN canaries in the padding lanes of the ragged last block (inputs and
    links) must not reach any output: every kernel variant reads only real
    sites, so the result equals the canary-free one bit for bit."""
    dims = (2, 4, 6, 6)  # 144 sites per parity: 16 padding lanes in the last block
    reps, precs = (hr.HR_FUND, hr.HR_ADJ), (hr.HR_F64, hr.HR_F32, hr.HR_F16)
    c = _forced_context(tmp_path, monkeypatch, "pad", dims, reps, precs, 1, variant, block)
    for rep in reps:
        nc = 2 if rep == hr.HR_FUND else 3
        q = synth.haar_links(dims, 41)
        psi = synth.gaussian_spinor(dims, nc, 42)
        for prec in precs:
            gauge = fields.pack_gauge(c, dims, rep, prec, fields.gauge_to_device(q))
            src = fields.pack_spinor(c, dims, rep, prec, hr.HR_ODD, fields.spinor_to_device(psi))
            outs = []
            for canary in (False, True):
                g, s = gauge.clone(), src.clone()
                if canary:
                    s[torch.as_tensor(_spinor_padding_bytes(dims, rep, prec), device="cuda")] = 0xFF
                    g[torch.as_tensor(_gauge_padding_bytes(dims, prec), device="cuda")] = 0xFF
                dst = fields.empty_spinor(dims, rep, prec, hr.HR_EVEN)
                hr.hr_dirac_eo(c, dims, -0.3, rep, prec, hr.HR_EVEN, hr.HR_OP_HOP, 1, g, s, dst)
                outs.append(fields.unpack_spinor(c, dims, rep, prec, hr.HR_EVEN, dst).cpu().numpy())
            assert np.all(np.isfinite(outs[1])), (rep, prec)
            assert np.array_equal(outs[0], outs[1]), (rep, prec)
    c.close()
