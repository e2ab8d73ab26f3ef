"""The value range of the FP64 class (pairs of floats) and the solvers'
source rescaling.

The packed FP64 layouts keep the float exponent range: a real keeps 48
significant bits while its low float is normal (|v| >= 2^-102) and an
operator's sums stay finite well below 2^128.  So (i) the pack kernels flag
NaN, Inf and magnitudes above 2^120, reported by hr_ctx_status and by the
solvers; (ii) the CG rescales each source by a power of two into [0.5, 1),
which is exact, so sources of magnitude 1e-20 or 1e20 (whose squared norms
leave the float range) solve like any other; (iii) a source whose largest
component is below 2^-100 has lost low bits in packing and is refused.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402

DIMS = (8, 8, 8, 8)
M0 = -0.2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


@pytest.fixture(scope="module")
def system(ctx):
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(DIMS, 1002), DIMS, 0.6)
    b = synth.gaussian_spinor(DIMS, 2, 2002)
    b[oracle.parity_mask(DIMS) == 1] = 0
    L = oracle.expand_links(DIMS, 2, q)
    xo, it, tr, ok = oracle.cg(DIMS, L, M0, b, tol=1e-12)
    assert ok
    gauge = fields.pack_gauge(ctx, DIMS, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    return {"q": q, "L": L, "b": b, "xo": xo, "gauge": gauge}


def solve(ctx, gauge, b, inner=hr.HR_F64):
    opts = hr.hr_solver_default_opts()
    opts.inner_prec = inner
    opts.reliable_delta = 0.1 if inner == hr.HR_F64 else 0.01
    bp = fields.pack_spinor(ctx, DIMS, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(DIMS, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(DIMS, hr.HR_FUND, opts))
    rc, _ = hr.hr_cg_solve(ctx, DIMS, M0, hr.HR_FUND, opts, gauge, bp, xp, work, raise_on_error=False)
    x = fields.unpack_spinor(ctx, DIMS, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
    return rc, x


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("scale", [1e-20, 1e20, 1e-28, 1e34])
def test_cg_source_scale_is_irrelevant(ctx, system, scale, inner):
    """Sources far from 1 (their squared norm outside the float range) solve
    to the true residual 1e-10 and to the oracle's solution, scaled."""
    b = system["b"] * scale
    rc, x = solve(ctx, system["gauge"], b, inner)
    assert rc == hr.HR_OK, hr.STATUS_NAMES.get(rc, rc)
    res = np.linalg.norm(b - oracle.normal(DIMS, system["L"], M0, x)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    even = oracle.parity_mask(DIMS) == 0
    xo = system["xo"] * scale
    assert np.linalg.norm((x - xo)[even]) / np.linalg.norm(xo[even]) < 1e-7


@pytest.mark.parametrize("inner", [hr.HR_F64, hr.HR_F16])
def test_cg_power_of_two_scaling_is_exact(ctx, system, inner):
    """Scaling b by 2^70 scales x by 2^70 bit for bit: the solver's internal
    rescaling makes the two solves the same arithmetic."""
    rc1, x1 = solve(ctx, system["gauge"], system["b"], inner)
    rc2, x2 = solve(ctx, system["gauge"], system["b"] * 2.0 ** 70, inner)
    assert rc1 == rc2 == hr.HR_OK
    assert np.array_equal(x2, x1 * 2.0 ** 70)


def test_tiny_components_next_to_large_ones_are_fine(ctx, system):
    """Small magnitudes are not flagged: only the field's largest component
    decides whether the pairs keep their precision."""
    b = system["b"].copy()
    b[::7] *= 1e-35
    bp = fields.pack_spinor(ctx, DIMS, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    hr.hr_ctx_status(ctx)
    del bp
    rc, x = solve(ctx, system["gauge"], b)
    assert rc == hr.HR_OK
    res = np.linalg.norm(b - oracle.normal(DIMS, system["L"], M0, x)) / np.linalg.norm(b)
    assert res <= 1e-10, res


def test_source_below_range_is_refused(ctx, system):
    rc, x = solve(ctx, system["gauge"], system["b"] * 1e-33)
    assert rc == hr.HR_ERR_UNSUPPORTED
    assert b"2^-100" in hr.lib().hr_last_error(ctx.handle)


@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32])
def test_pack_flags_values_above_range(ctx, system, prec):
    b = system["b"].copy()
    b[0, 1, 0] = 3e37  # site 0 is even
    fields.pack_spinor(ctx, DIMS, hr.HR_FUND, prec, hr.HR_EVEN, fields.spinor_to_device(b))
    with pytest.raises(hr.HrError) as e:
        hr.hr_ctx_status(ctx)
    assert e.value.code == hr.HR_ERR_UNSUPPORTED
    hr.hr_ctx_status(ctx)  # the flags were cleared
    # the solver makes the same check before it starts
    rc, _ = solve(ctx, system["gauge"], b)
    assert rc == hr.HR_ERR_UNSUPPORTED
    assert b"2^120" in hr.lib().hr_last_error(ctx.handle)
    hr.hr_ctx_status(ctx)


def test_pack_flags_non_finite_values(ctx, system):
    b = system["b"].copy()
    b[2, 2, 1] = np.nan  # site 2 is even
    fields.pack_spinor(ctx, DIMS, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    with pytest.raises(hr.HrError) as e:
        hr.hr_ctx_status(ctx)
    assert e.value.code == hr.HR_ERR_NUMERIC
    q = system["q"].copy()
    q[1, 7, 2] = np.inf
    fields.pack_gauge(ctx, DIMS, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    with pytest.raises(hr.HrError) as e:
        hr.hr_ctx_status(ctx)
    assert e.value.code == hr.HR_ERR_NUMERIC
    hr.hr_ctx_status(ctx)
