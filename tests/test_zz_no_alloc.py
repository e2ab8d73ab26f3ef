"""The allocation-free norm entry point, hr_norm2_noalloc.

Who needs it: a caller that may not allocate device memory -- for example a
host application that reserves the whole GPU for its own memory pool up front,
or a plug-in that must not touch the process's CUDA allocator -- cannot create
an hr_ctx, because context creation calls cudaMalloc for the reduction
scratch.  hr_norm2_noalloc needs no context: its scratch is a fixed array
inside the library.  This file checks, through the C ABI, that it returns
|v|^2 as summed on the host from the canonical field (and the same as the
context-based hr_norm2), on two calls in a row (the second call must not be
disturbed by what the first one left in the shared scratch), and that after
the first call on the device a call takes no device memory.  The file is
named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import hr, fields  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def even_sites(dims):
    x = np.indices(dims).sum(axis=0).reshape(-1)
    return (x & 1) == 0


def noalloc(dims, rep, n_rhs, v, result):
    L = hr.lib()
    return L.hr_norm2_noalloc(hr.lattice(dims), rep, n_rhs, hr._ptr(v), hr._ptr(result),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (6, 4, 2, 6), (16, 16, 16, 16)])
def test_noalloc_norm_matches_context_norm_twice(ctx, rep, dims):
    nc = 2 if rep == hr.HR_FUND else 3
    psi = synth.gaussian_spinor(dims, nc, 77)
    packed = fields.pack_spinor(ctx, dims, rep, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(psi))
    even = even_sites(dims)
    want = float(np.sum(np.abs(psi[even]) ** 2))
    lib_norm = hr.hr_norm2(ctx, dims, rep, packed)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        assert noalloc(dims, rep, 1, packed, out) == hr.HR_OK
        torch.cuda.synchronize()
        got = out.item()
        # the packed pairs hold 48 significant bits: 1e-13 relative
        assert abs(got - want) <= 1e-13 * want, (got, want)
        assert abs(got - lib_norm) <= 1e-13 * want, (got, lib_norm)


def test_noalloc_norm_multi_rhs(ctx):
    dims = (4, 6, 2, 6)
    n = 4
    psis = synth.gaussian_spinor(dims, 2, 78, n_rhs=n)
    packed = fields.pack_spinor(ctx, dims, hr.HR_FUND, hr.HR_F64, hr.HR_ODD, fields.spinor_to_device(psis))
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    odd = ~even_sites(dims)
    for _ in range(2):
        assert noalloc(dims, hr.HR_FUND, n, packed, out) == hr.HR_OK
        torch.cuda.synchronize()
        for r in range(n):
            want = float(np.sum(np.abs(psis[r][odd]) ** 2))
            assert abs(out[r].item() - want) <= 1e-13 * want


def test_noalloc_rejects_what_does_not_fit(ctx):
    dims = (4, 4, 4, 4)
    v = fields.zeros_spinor(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN)
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert noalloc(dims, hr.HR_FUND, 64, v, out) == hr.HR_ERR_WORKSPACE
    assert noalloc(dims, hr.HR_FUND, 3, v, out) == hr.HR_ERR_UNSUPPORTED
    assert noalloc((4, 4, 4, 3), hr.HR_FUND, 1, v, out) == hr.HR_ERR_UNSUPPORTED
    assert noalloc(dims, hr.HR_FUND, 1, None, out) == hr.HR_ERR_INVALID_ARG
    # boundary bits and twist angles are checked as by every other entry point
    assert noalloc(hr.Lattice(dims, 16), hr.HR_FUND, 1, v, out) == hr.HR_ERR_INVALID_ARG
    assert noalloc(hr.Lattice(dims, 0, (float("nan"), 0, 0, 0)), hr.HR_FUND, 1, v, out) == hr.HR_ERR_INVALID_ARG
    assert noalloc((4, 4, 4, 0), hr.HR_FUND, 1, v, out) == hr.HR_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0)


def test_noalloc_takes_no_device_memory_after_its_first_call(ctx):
    """The first call on a device sets up the fixed array (under lazy module
    loading the driver places it then); every later call leaves the free
    device memory exactly as it was."""
    dims = (8, 8, 8, 8)
    psi = synth.gaussian_spinor(dims, 2, 79)
    packed = fields.pack_spinor(ctx, dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, fields.spinor_to_device(psi))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert noalloc(dims, hr.HR_FUND, 1, packed, out) == hr.HR_OK  # warm-up: the set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert noalloc(dims, hr.HR_FUND, 1, packed, out) == hr.HR_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
