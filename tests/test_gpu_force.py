"""Link derivatives on the GPU (su(2) force and quaternion gradient) vs the oracle."""

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


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 6, 2, 6), (8, 4, 6, 4)])
def test_force_and_link_grad_match_oracle(ctx, dims):
    q = synth.haar_links(dims, 51)
    a = synth.gaussian_spinor(dims, 2, 52)
    b = synth.gaussian_spinor(dims, 2, 53)
    L = oracle.expand_links(dims, 2, q)
    gauge = fields.pack_gauge(ctx, dims, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    ap = fields.pack_spinor(ctx, dims, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(a))
    bp = fields.pack_spinor(ctx, dims, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, fields.spinor_to_device(b))
    V = int(np.prod(dims))
    F = torch.zeros((4, V, 3), dtype=torch.float64, device="cuda")
    hr.hr_force(ctx, dims, gauge, ap, bp, 1.0, F)
    want = oracle.force(dims, L, a, b)
    got = F.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-13
    # beta accumulates
    hr.hr_force(ctx, dims, gauge, ap, bp, -0.5, F)
    np.testing.assert_allclose(F.cpu().numpy(), 0.5 * want, rtol=0, atol=1e-12 * np.abs(want).max())
    G = torch.zeros((4, V, 4), dtype=torch.float64, device="cuda")
    hr.hr_link_grad(ctx, dims, ap, bp, 1.0, G)
    wantg = oracle.link_grad(dims, a, b)
    assert np.linalg.norm(G.cpu().numpy() - wantg) / np.linalg.norm(wantg) <= 1e-13
