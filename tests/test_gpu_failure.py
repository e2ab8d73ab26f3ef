"""Failure detection without a GPU fault: the tiled hop's only device wait
(its bulk copy landing on an mbarrier) is made to run out by a test-only
injection that announces the copy but never queues it.  The bounded wait must
give up, the kernel must fall back to global memory and raise the device error
flag, the solver must report HR_ERR_TIMEOUT, and the device must stay usable."""

import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402


def _solve(c, dims, q, b):
    opts = hr.hr_solver_default_opts()
    gauge = fields.pack_gauge(c, dims, hr.HR_FUND, hr.HR_F64, fields.gauge_to_device(q))
    bp = fields.pack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(b))
    xp = fields.zeros_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    work = fields.empty_bytes(hr.hr_cg_workspace_bytes(dims, hr.HR_FUND, opts))
    rc, info = hr.hr_cg_solve(c, dims, 0.1, hr.HR_FUND, opts, gauge, bp, xp, work, raise_on_error=False)
    x = fields.unpack_spinor(c, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xp).cpu().numpy()
    return rc, info, x


def test_tiled_copy_timeout_is_reported_and_recovered(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims = (4, 4, 8, 8)  # 512 sites per parity: 8 tiles of 64 sites
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({f"hop:r0:p0:{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}:n1": [8, 64]}))
    monkeypatch.setenv("HR_AUTOTUNE_CACHE", str(cache))
    q = synth.haar_links(dims, 601)
    b = synth.gaussian_spinor(dims, 2, 602)
    b[oracle.parity_mask(dims) == 1] = 0
    L = oracle.expand_links(dims, 2, q)

    monkeypatch.setenv("HR_INJECT_TILE_NO_COPY", "1")
    c = hr.Context(0)
    assert hr.hr_tune_lookup(c, dims, hr.HR_FUND, hr.HR_F64) == (8, 64)
    rc, info, x = _solve(c, dims, q, b)
    assert rc == hr.HR_ERR_TIMEOUT
    assert "did not land" in c.last_error()
    # the waits fell back to global memory: the arithmetic is still right
    res = np.linalg.norm(b - oracle.normal(dims, L, 0.1, x)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    c.close()

    monkeypatch.delenv("HR_INJECT_TILE_NO_COPY")
    c2 = hr.Context(0)
    rc2, info2, x2 = _solve(c2, dims, q, b)
    assert rc2 == hr.HR_OK
    assert np.array_equal(x, x2)
    c2.close()
