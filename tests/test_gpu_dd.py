"""The hop of a lattice split along time into slabs (the multi-GPU data flow,
all slabs on one GPU; the exchange a device copy between slabs), against the
FP64 oracle's hop of the whole lattice and against the library's own hop of
the whole lattice.

Cases: 1, 2, 3, 4 and 6 slabs, slabs of 2 slices (both faces of a slab are
neighbours of each other's sites), every representation and precision, both
output parities, periodic, antiperiodic-in-time (the sign sits on the last
slab's links only) and antiperiodic in time and x3.  Tolerances as for the
whole-lattice hop (FP64 1e-13, FP32 1e-6, FP16 4e-3 relative L2).
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import dd, hr, fields  # noqa: E402

TOL = {hr.HR_F64: 1e-13, hr.HR_F32: 1e-6, hr.HR_F16: 4e-3}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hr.Context(0)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


CASES = [((8, 4, 6, 6), 1), ((8, 4, 6, 6), 2), ((8, 4, 6, 6), 4), ((12, 4, 2, 6), 3), ((12, 4, 2, 6), 6)]


@pytest.mark.parametrize("bc", [0, 1, 9])
@pytest.mark.parametrize("prec", [hr.HR_F64, hr.HR_F32, hr.HR_F16])
@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ, hr.HR_ADJ_MAT])
@pytest.mark.parametrize("dims,n", CASES, ids=[f"{d[0]}x{d[1]}x{d[2]}x{d[3]}_n{n}" for d, n in CASES])
def test_slab_hop_matches_oracle(ctx, dims, n, rep, prec, bc):
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, 401)
    psi = synth.gaussian_spinor(dims, nc, 402)
    L = oracle.expand_links(dims, nc, q)
    slabs = dd.TimeSlabs(dims, n, bc)
    op = dd.SlabHop(ctx, slabs, rep, prec, q)
    for p in (hr.HR_EVEN, hr.HR_ODD):
        got = op.hop(p, psi)
        want = -0.5 * oracle.hop(dims, L, psi, parity=p, bc=bc)
        m = oracle.parity_mask(dims) == p
        assert rel(got[m], want[m]) <= TOL[prec], (p, rel(got[m], want[m]))
        assert np.all(got[~m] == 0)


@pytest.mark.parametrize("rep", [hr.HR_FUND, hr.HR_ADJ])
def test_slab_hop_equals_whole_lattice_hop(ctx, rep):
    """FP64: the slab hop and the library's whole-lattice hop differ only by
    the rounding of the face terms (subtracted and added back): a few units of
    the pairs' 2^-48 = 3.6e-15 (measured 4.9e-15 fundamental, 5.9e-15 adjoint)."""
    dims, n, bc = (16, 6, 4, 8), 4, 1
    nc = 2 if rep == hr.HR_FUND else 3
    q = synth.haar_links(dims, 411)
    psi = synth.gaussian_spinor(dims, nc, 412)
    lat = hr.Lattice(dims, bc)
    gauge = fields.pack_gauge(ctx, lat, rep, hr.HR_F64, fields.gauge_to_device(q))
    op = dd.SlabHop(ctx, dd.TimeSlabs(dims, n, bc), rep, hr.HR_F64, q)
    for p in (hr.HR_EVEN, hr.HR_ODD):
        src = fields.pack_spinor(ctx, lat, rep, hr.HR_F64, 1 - p, fields.spinor_to_device(psi))
        dst = fields.empty_spinor(lat, rep, hr.HR_F64, p)
        hr.hr_dirac_eo(ctx, lat, 0.0, rep, hr.HR_F64, p, hr.HR_OP_HOP, 1, gauge, src, dst)
        whole = fields.unpack_spinor(ctx, lat, rep, hr.HR_F64, p, dst).cpu().numpy()
        m = oracle.parity_mask(dims) == p
        assert rel(op.hop(p, psi)[m], whole[m]) <= 1e-14


def test_face_bytes_and_bad_arguments(ctx):
    local = hr.Lattice((4, 4, 6, 6))
    nf = 4 * 6 * 6 // 2
    assert hr.hr_dd_face_bytes(local, hr.HR_FUND, hr.HR_F64) == (nf * 8 * 8 + 255) // 256 * 256
    assert hr.hr_dd_face_bytes(local, hr.HR_ADJ, hr.HR_F32) == (nf * 12 * 4 + 255) // 256 * 256
    assert hr.hr_dd_face_bytes((4, 4, 6, 5), hr.HR_FUND, hr.HR_F64) == 0
    g = fields.empty_bytes(hr.hr_gauge_packed_bytes(local, 0, 0))
    s = fields.zeros_spinor(local, 0, 0, hr.HR_EVEN)
    f1 = fields.empty_bytes(hr.hr_dd_face_bytes(local, 0, 0))
    f2 = fields.empty_bytes(hr.hr_dd_face_bytes(local, 0, 0))
    L = hr.lib()
    st = torch.cuda.current_stream().cuda_stream
    tw = hr.Lattice((4, 4, 6, 6), 0, (0.3, 0, 0, 0))
    assert L.hr_dd_pack_faces(ctx.handle, hr.lattice(tw), 0, 0, 0, g.data_ptr(), s.data_ptr(), f1.data_ptr(),
                              f2.data_ptr(), st) == hr.HR_ERR_UNSUPPORTED
    assert L.hr_dd_pack_faces(ctx.handle, hr.lattice(local), 0, 0, 0, g.data_ptr(), s.data_ptr(), f1.data_ptr(),
                              f1.data_ptr(), st) == hr.HR_ERR_INVALID_ARG
    assert L.hr_dd_hop_boundary(ctx.handle, hr.lattice(local), 0, 0, 2, g.data_ptr(), s.data_ptr(), f1.data_ptr(),
                                f2.data_ptr(), s.data_ptr(), st) == hr.HR_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        dd.TimeSlabs((8, 4, 4, 4), 3)   # 8 slices do not split into 3 slabs
    with pytest.raises(ValueError):
        dd.TimeSlabs((12, 4, 4, 4), 4)  # slabs of 3 slices: odd
