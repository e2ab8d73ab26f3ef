"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and its size/argument logic behaves as documented (no GPU needed)."""

import ctypes
import os
import re

import pytest

from paper_2411_18511_gb300 import hr

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "hirep_gb300.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(hr_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_binding_list():
    assert declared_functions() == sorted(hr.EXPORTED)


def test_library_exports_every_declared_symbol():
    L = hr.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert hr.hr_version().startswith("hirep_gb300")


def test_mass_conventions():
    for kappa in (0.12, 0.125, 1 / 7.6, 0.2):
        m0 = hr.hr_kappa_to_m0(kappa)
        assert abs(m0 - (1 / (2 * kappa) - 4)) < 1e-15
        assert abs(hr.hr_m0_to_kappa(m0) - kappa) < 1e-15
    assert abs(hr.hr_m0_to_kappa(-0.2) - 1 / 7.6) < 1e-15


def test_packed_sizes():
    dims = (4, 6, 2, 6)  # V_h = 144 sites: 5 blocks of 32, the last ragged
    nblk = (144 + 31) // 32
    assert hr.hr_spinor_packed_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1) == nblk * 32 * 128
    assert hr.hr_spinor_packed_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, 1) == 2 * nblk * 32 * 128
    assert hr.hr_spinor_packed_bytes(dims, hr.HR_ADJ, hr.HR_F32, hr.HR_ODD, 1) == nblk * 32 * 96
    f16 = nblk * 32 * 32 + nblk * 32 * 4
    assert hr.hr_spinor_packed_bytes(dims, hr.HR_FUND, hr.HR_F16, hr.HR_ODD, 1) == (f16 + 255) // 256 * 256
    nb4 = (144 * 4 + 31) // 32
    assert hr.hr_spinor_packed_bytes(dims, hr.HR_FUND, hr.HR_F32, hr.HR_EVEN, 4) == nb4 * 32 * 64
    assert hr.hr_gauge_packed_bytes(dims, hr.HR_FUND, hr.HR_F64) == 8 * nblk * 32 * 32
    assert hr.hr_gauge_packed_bytes(dims, hr.HR_ADJ, hr.HR_F32) == 8 * nblk * 32 * 16
    assert hr.hr_gauge_packed_bytes(dims, hr.HR_ADJ_MAT, hr.HR_F64) == 8 * nblk * 32 * 72
    assert hr.hr_dirac_workspace_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_OP_HOP) == 0
    assert hr.hr_dirac_workspace_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_OP_NORMAL) == 2 * nblk * 32 * 128


@pytest.mark.parametrize("dims", [(4, 4, 4, 3), (1, 4, 4, 4), (0, 2, 2, 2), (4, 4, 4, -2)])
def test_invalid_lattices_have_no_size(dims):
    assert hr.hr_spinor_packed_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1) == 0
    assert hr.hr_gauge_packed_bytes(dims, hr.HR_FUND, hr.HR_F64) == 0


def test_boundary_bits():
    """hr_lattice.bc: one antiperiodic bit per direction; other bits make the lattice invalid."""
    d = (4, 4, 4, 4)
    base = hr.hr_gauge_packed_bytes(d, hr.HR_FUND, hr.HR_F64)
    for bc in (1, 9, 15):
        lat = hr.Lattice(d, bc)
        assert lat == d and lat.bc == bc
        assert hr.lattice(lat).bc == bc
        assert hr.hr_gauge_packed_bytes(lat, hr.HR_FUND, hr.HR_F64) == base
    assert hr.HR_BC_ANTIPERIODIC(0) == 1 and hr.HR_BC_ANTIPERIODIC(3) == 8
    assert hr.lattice(d).bc == 0
    for bc in (16, -1, 255):
        assert hr.hr_gauge_packed_bytes(hr.Lattice(d, bc), hr.HR_FUND, hr.HR_F64) == 0
        assert hr.hr_spinor_packed_bytes(hr.Lattice(d, bc), hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1) == 0


def test_invalid_enums_and_rhs_have_no_size():
    d = (4, 4, 4, 4)
    assert hr.hr_spinor_packed_bytes(d, 5, hr.HR_F64, hr.HR_EVEN, 1) == 0
    assert hr.hr_spinor_packed_bytes(d, hr.HR_FUND, 9, hr.HR_EVEN, 1) == 0
    assert hr.hr_spinor_packed_bytes(d, hr.HR_FUND, hr.HR_F64, 3, 1) == 0
    for n in (0, 3, 64):
        assert hr.hr_spinor_packed_bytes(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, n) == 0


def test_solver_defaults_and_workspace():
    o = hr.hr_solver_default_opts()
    assert o.tol == 1e-10 and o.maxiter == 20000 and o.inner_prec == hr.HR_F64
    assert o.reliable_delta == 0.1 and o.n_rhs == 1 and o.x0_is_guess == 0
    d = (8, 8, 8, 8)
    w64 = hr.hr_cg_workspace_bytes(d, hr.HR_FUND, o)
    # r, p, q and two operator temporaries, and the rescaled copy of b
    assert w64 == 6 * hr.hr_spinor_packed_bytes(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1)
    o.inner_prec = hr.HR_F16
    assert hr.hr_cg_workspace_bytes(d, hr.HR_FUND, o) > 0
    o.n_rhs = 3
    assert hr.hr_cg_workspace_bytes(d, hr.HR_FUND, o) == 0


def test_hmc_and_clover_force_workspaces():
    """Host-side sizes (no device needed): each HMC option adds its buffers."""
    d = (8, 8, 8, 8)
    V = 8 ** 4
    half = hr.hr_spinor_packed_bytes(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1)
    assert hr.hr_clover_force_workspace_bytes(d) == V * 48 * 8 + 5 * half
    assert hr.hr_clover_force_workspace_bytes((8, 8, 8, 7)) == 0
    prm = hr.hr_hmc_params_default(2.2, 0.1, True, 4, 1.0)
    base = hr.hr_hmc_workspace_bytes(d, prm)
    assert base > 0
    prm.n_steps_gauge = 3                     # a second force buffer
    two = hr.hr_hmc_workspace_bytes(d, prm)
    assert two - base == 12 * V * 8
    prm.clover, prm.c_sw = 1, 1.0             # the clover field and the force workspace
    clov = hr.hr_hmc_workspace_bytes(d, prm)
    cfield = hr.hr_clover_packed_bytes(d, hr.HR_FUND, hr.HR_F64)
    assert clov - two >= cfield + hr.hr_clover_force_workspace_bytes(d)
    prm.hasenbusch, prm.m0_hasenbusch = 1, 0.5  # a heavy clover field and the ratio term's fields
    assert hr.hr_hmc_workspace_bytes(d, prm) - clov >= cfield + 4 * half


def test_null_context_is_rejected():
    L = hr.lib()
    assert L.hr_last_error(None) == b"null context"
    assert L.hr_ctx_destroy(None) == hr.HR_ERR_INVALID_ARG
    rc = L.hr_dirac_eo(None, hr.lattice((4, 4, 4, 4)), 0.0, 0, 0, 0, 0, 1, None, None, None, None, 0, None)
    assert rc == hr.HR_ERR_INVALID_ARG


def test_context_creation_matches_device_presence():
    import torch
    h = ctypes.c_void_p()
    rc = hr.lib().hr_ctx_create(ctypes.byref(h), 0)
    if torch.cuda.is_available():
        assert rc == hr.HR_OK
        hr.lib().hr_ctx_destroy(h)
    else:
        assert rc == hr.HR_ERR_CUDA and not h.value
    rc = hr.lib().hr_ctx_create(ctypes.byref(h), 999)
    assert rc == hr.HR_ERR_CUDA
