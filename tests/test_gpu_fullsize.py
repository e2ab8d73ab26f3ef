"""Parity at the benchmarked sizes, in the launch shapes the benchmark uses.

The small-lattice tests cover every kernel variant, but three launch paths are
only taken at full size: the 32^4 solves (the 128-thread hop fills the
4096-block cap of the reducing launches), the 24^4 x 32 right-hand-side
solve (the reducing launches run grid-stride loops over 5.3 M virtual sites)
and the 48^4 hops of every representation in the shape the autotuner picks.
Here each is checked against the FP64 oracle:

* 48^4 hop D_eo / D_oe (both parities), fundamental and adjoint (quaternion
  links rebuilt in registers, and stored 3x3 matrices), FP64 and FP32, on
  2000 random output sites plus both ends of each parity, after the same
  autotuning call the benchmark makes; and the fundamental FP64 hop in every
  launch shape the tuner can choose, forced through the tuning cache.
  Tolerances as in the small-lattice tests: FP64 1e-13, FP32 1e-6 relative L2.
* 32^4 CG on Mhat^+ Mhat (smeared links, plaquette 0.6, m0 = -0.2, tol 1e-10),
  FP64 and FP32 / FP16 inner solvers at every reliable_delta the benchmark
  sweeps: the true residual |b - A x| / |b| recomputed by the oracle <= 1e-10,
  the FP64 iteration count within 2 of the oracle CG's, and the distance to
  the oracle CG's solution (bounded by cond(A) x tol; gated loosely).
* 24^4 CG with 32 right-hand sides (FP32 inner, FP64 reliable updates): the
  oracle's true residual of every right-hand side, and the distance to the
  oracle CG's solution for the first and the last one (each oracle CG takes
  seconds of host time).
"""

import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6}
D48 = (48, 48, 48, 48)
D32 = (32, 32, 32, 32)
D24 = (24, 24, 24, 24)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def sample_sites(dims, parity, n=2000, seed=7):
    cand = np.where(oracle.parity_mask(dims) == parity)[0]
    rng = np.random.default_rng(seed + parity)
    return np.concatenate([cand[:16], cand[-16:], rng.choice(cand, n, replace=False)])


# ---------------------------------------------------------------------- 48^4 hops

@pytest.fixture(scope="module")
def fields48():
    """The benchmark's 48^4 inputs: links seed 1003, fundamental source seed
    2003, adjoint source seed 2004."""
    q = synth.haar_links(D48, 1003)
    return {"q": q, "psi2": synth.gaussian_spinor(D48, 2, 2003), "psi3": synth.gaussian_spinor(D48, 3, 2004)}


@pytest.fixture(scope="module")
def links48(fields48):
    cache = {}

    def get(nc):
        if nc not in cache:
            cache.clear()  # one colour-matrix field at a time (3 GB for the adjoint)
            cache[nc] = oracle.expand_links(D48, nc, fields48["q"])
        return cache[nc]
    return get


def hop48_errors(c, rep, prec, gauge, dpsi, psi, L):
    """Relative L2 error of -1/2 H at the sampled sites of both parities."""
    errs = []
    for out_par in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(c, D48, rep, prec, 1 - out_par, dpsi)
        dst = fields.empty_spinor(D48, rep, prec, out_par)
        hr.hr_dirac_eo(c, D48, 0.0, rep, prec, out_par, hr.HR_OP_HOP, 1, gauge, src, dst)
        sites = sample_sites(D48, out_par)
        full = fields.unpack_spinor(c, D48, rep, prec, out_par, dst)
        got = full[torch.as_tensor(sites, device=full.device)].cpu().numpy()
        del full, src, dst
        want = -0.5 * oracle.hop_sites(D48, L, psi, sites)
        errs.append(rel(got, want))
    return errs


@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT])
def test_hop_48_tuned_shape(ctx, fields48, links48, rep, prec):
    """The 48^4 hop of each representation and precision after the autotuning
    call the benchmark makes (reps = 10), in whatever shape it chose."""
    nc = 2 if rep == hr.HR_FUND else 3
    psi = fields48["psi2"] if nc == 2 else fields48["psi3"]
    gauge = fields.pack_gauge(ctx, D48, rep, prec, fields.gauge_to_device(fields48["q"]))
    dpsi = fields.spinor_to_device(psi)
    src = fields.pack_spinor(ctx, D48, rep, prec, hr.HR_ODD, dpsi)
    dst = fields.empty_spinor(D48, rep, prec, hr.HR_EVEN)
    res = hr.hr_autotune_hop(ctx, D48, rep, prec, hr.HR_EVEN, 1, gauge, src, dst, reps=10)
    del src, dst
    assert hr.hr_tune_lookup(ctx, D48, rep, prec) == (res.variant, res.block)
    errs = hop48_errors(ctx, rep, prec, gauge, dpsi, psi, links48(nc))
    print(f"rep {rep} prec {prec} tuned (variant {res.variant}, block {res.block}): errors {errs}")
    assert max(errs) <= TOL[prec], (res.variant, res.block, errs)


def _fund_f64_shapes():
    return [(v, b) for v in range(14) for b in (64, 128, 192, 256)]


@pytest.fixture(scope="module")
def fund48_f64(ctx, fields48):
    gauge = fields.pack_gauge(ctx, D48, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(fields48["q"]))
    return gauge, fields.spinor_to_device(fields48["psi2"])


@pytest.mark.parametrize("variant,block", _fund_f64_shapes())
def test_hop_48_fund_f64_forced_shape(tmp_path, monkeypatch, fields48, links48, fund48_f64, variant, block):
    """The benchmark's kernel (48^4 fundamental FP64) in every launch shape the
    tuner may choose, each forced through HR_AUTOTUNE_CACHE."""
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({f"hop:r0:p0:48x48x48x48:n1": [variant, block]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    c = hr.Context(0)
    try:
        assert hr.hr_tune_lookup(c, D48, hr.HR_FUND, hr.HR_F64) == (variant, block)
        gauge, dpsi = fund48_f64
        errs = hop48_errors(c, hr.HR_FUND, hr.HR_F64, gauge, dpsi, fields48["psi2"], links48(2))
        assert max(errs) <= 1e-13, errs
    finally:
        c.close()


# ---------------------------------------------------------------------- 32^4 CG

@pytest.fixture(scope="module")
def cg32(ctx):
    """The benchmark's 32^4 system: APE-smeared Haar links (seed 1002) at
    plaquette 0.6, Gaussian even source (seed 2002), m0 = -0.2; the hop shapes
    tuned for the three precisions the solvers use; the oracle CG's solution."""
    q, _, plaq = synth.ape_smear_to_plaquette(synth.haar_links(D32, 1002), D32, 0.6)
    assert abs(plaq - 0.6) < 2e-3
    b = synth.gaussian_spinor(D32, 2, 2002)
    b[oracle.parity_mask(D32) == 1] = 0
    bdev = fields.spinor_to_device(b)
    for prec in (hr.HR_F64, hr.HR_F32, hr.HR_F16):
        gp = fields.pack_gauge(ctx, D32, hr.HR_FUND, prec, fields.gauge_to_device(q))
        src = fields.pack_spinor(ctx, D32, hr.HR_FUND, prec, hr.HR_ODD, bdev)
        dst = fields.empty_spinor(D32, hr.HR_FUND, prec, hr.HR_EVEN)
        hr.hr_autotune_hop(ctx, D32, hr.HR_FUND, prec, hr.HR_EVEN, 1, gp, src, dst, reps=10)
        del gp, src, dst
    L = oracle.expand_links(D32, 2, q)
    xo, it, tr, ok = oracle.cg(D32, L, -0.2, b, tol=1e-10)
    assert ok and tr <= 1e-10
    gauge = fields.pack_gauge(ctx, D32, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(ctx, D32, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, bdev)
    return {"q": q, "L": L, "b": b, "xo": xo, "iters": it, "gauge": gauge, "bp": bp}


@pytest.mark.parametrize("inner,delta", [(hr.HR_F64, 0.1), (hr.HR_F32, 0.1), (hr.HR_F32, 1e-2), (hr.HR_F32, 1e-3),
                                         (hr.HR_F32, 1e-4), (hr.HR_F32, 1e-5),
                                         (hr.HR_F16, 0.1), (hr.HR_F16, 3e-2), (hr.HR_F16, 1e-2)])
def test_cg_32_matches_oracle(ctx, cg32, inner, delta):
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    opts.reliable_delta = delta
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(D32, hr.HR_FUND, opts))
    xp = fields.zeros_spinor(D32, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    rc, info = hr.hr_cg_solve(ctx, D32, -0.2, hr.HR_FUND, opts, cg32["gauge"], cg32["bp"], xp, work)
    assert rc == hr.HR_OK, (rc, info.true_rel_residual)
    x = fields.unpack_spinor(ctx, D32, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
    b = cg32["b"]
    res = np.linalg.norm(b - oracle.normal(D32, cg32["L"], -0.2, x)) / np.linalg.norm(b)
    even = oracle.parity_mask(D32) == 0
    err = rel(x[even], cg32["xo"][even])
    print(f"inner {inner} delta {delta}: iters {info.iters} (oracle {cg32['iters']}), reliable "
          f"{info.n_reliable_updates}, oracle residual {res:.3e}, library residual {info.true_rel_residual:.3e}, "
          f"|x - x_oracle| / |x_oracle| {err:.3e}")
    assert res <= 1e-10, res
    assert abs(res - info.true_rel_residual) <= 1e-11
    if inner == hr.HR_F64:
        assert abs(info.iters - cg32["iters"]) <= 2, (info.iters, cg32["iters"])
    assert err < 1e-6, err


# ---------------------------------------------------------------------- 24^4 x 32 RHS

@pytest.mark.parametrize("delta", [0.1, 1e-5])
def test_cg_24_multi_rhs_32_matches_oracle(ctx, delta):
    """The multi-RHS configuration: 24^4 smeared links (seed 1004), 32 Gaussian
    sources (seed 2004), FP32 inner / FP64 outer CG with the hop shapes tuned
    for 32 right-hand sides, at the default reliable_delta and at the
    benchmark's, every right-hand side checked by the oracle."""
    n = 32
    q, _, plaq = synth.ape_smear_to_plaquette(synth.haar_links(D24, 1004), D24, 0.6)
    bs = synth.gaussian_spinor(D24, 2, 2004, n_rhs=n)
    odd = oracle.parity_mask(D24) == 1
    bs[:, odd] = 0
    dev = fields.spinor_to_device(bs)
    gauge = fields.pack_gauge(ctx, D24, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    for tp in (hr.HR_F32, hr.HR_F64):
        gp = fields.pack_gauge(ctx, D24, hr.HR_FUND, tp, fields.gauge_to_device(q))
        ts = fields.pack_spinor(ctx, D24, hr.HR_FUND, tp, hr.HR_ODD, dev)
        td = fields.empty_spinor(D24, hr.HR_FUND, tp, hr.HR_EVEN, n)
        hr.hr_autotune_hop(ctx, D24, hr.HR_FUND, tp, hr.HR_EVEN, n, gp, ts, td, reps=10)
        del gp, ts, td
    bp = fields.pack_spinor(ctx, D24, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, dev)
    del dev
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = hr.HR_F32
    opts.reliable_delta = delta
    opts.n_rhs = n
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(D24, hr.HR_FUND, opts))
    xp = fields.zeros_spinor(D24, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, n)
    rc, info = hr.hr_cg_solve(ctx, D24, -0.2, hr.HR_FUND, opts, gauge, bp, xp, work)
    assert rc == hr.HR_OK, info.true_rel_residual
    xs = fields.unpack_spinor(ctx, D24, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp, n).cpu().numpy()
    L = oracle.expand_links(D24, 2, q)
    worst_res, worst_err = 0.0, 0.0
    for r in range(n):
        res = np.linalg.norm(bs[r] - oracle.normal(D24, L, -0.2, xs[r])) / np.linalg.norm(bs[r])
        worst_res = max(worst_res, res)
        assert res <= 1e-10, (r, res)
        assert np.all(xs[r][odd] == 0)
    for r in (0, n - 1):
        xo, it, tr, ok = oracle.cg(D24, L, -0.2, bs[r], tol=1e-10)
        assert ok
        err = rel(xs[r][~odd], xo[~odd])
        worst_err = max(worst_err, err)
        assert err < 1e-6, (r, err)
    print(f"24^4 x 32: iters {info.iters}, worst oracle residual {worst_res:.3e}, library max "
          f"{info.true_rel_residual:.3e}, worst |x - x_oracle| / |x_oracle| {worst_err:.3e}")
    assert abs(worst_res - info.true_rel_residual) <= 1e-11
