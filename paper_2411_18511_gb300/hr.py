"""ctypes binding of libhirep_gb300.so (argument marshalling only).

Every function here has the name of the C entry point it calls
(``include/hirep_gb300.h``) and only converts arguments: torch tensors become
device pointers, streams become ``cudaStream_t`` handles, status codes become
:class:`HrError`.  All computation happens in the library's CUDA kernels.
The library is built in-tree (``paper_2411_18511_gb300/_build``); if it cannot
be built or loaded, :func:`lib` raises -- there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import _build

# ------------------------------------------------------------------ enums
HR_OK, HR_ERR_INVALID_ARG, HR_ERR_UNSUPPORTED, HR_ERR_CUDA = 0, 1, 2, 3
HR_ERR_NOT_CONVERGED, HR_ERR_NUMERIC, HR_ERR_TIMEOUT, HR_ERR_WORKSPACE = 4, 5, 6, 7
HR_FUND, HR_ADJ, HR_ADJ_MAT = 0, 1, 2
HR_F64, HR_F32, HR_F16 = 0, 1, 2
HR_EVEN, HR_ODD, HR_FULL = 0, 1, 2
HR_OP_HOP, HR_OP_SCHUR, HR_OP_SCHUR_DAG, HR_OP_NORMAL = 0, 1, 2, 3
HR_SYSTEM_D, HR_SYSTEM_DDAG_D = 0, 1
HR_CLOVER_SW, HR_CLOVER_EXP = 0, 1
HR_INTEGRATOR_LEAPFROG, HR_INTEGRATOR_OMELYAN = 0, 1


def HR_BC_ANTIPERIODIC(mu: int) -> int:
    """Bit of ``hr_lattice.bc`` that makes direction mu (0 = time) antiperiodic."""
    return 1 << int(mu)


STATUS_NAMES = {0: "HR_OK", 1: "HR_ERR_INVALID_ARG", 2: "HR_ERR_UNSUPPORTED", 3: "HR_ERR_CUDA",
                4: "HR_ERR_NOT_CONVERGED", 5: "HR_ERR_NUMERIC", 6: "HR_ERR_TIMEOUT",
                7: "HR_ERR_WORKSPACE"}

# every symbol the header declares (checked by the ABI tests)
EXPORTED = [
    "hr_ctx_create", "hr_ctx_destroy", "hr_last_error", "hr_version", "hr_kappa_to_m0",
    "hr_m0_to_kappa", "hr_gauge_packed_bytes", "hr_spinor_packed_bytes", "hr_gauge_pack",
    "hr_spinor_pack", "hr_spinor_unpack", "hr_dirac_workspace_bytes", "hr_dirac_apply",
    "hr_dirac_eo", "hr_solver_default_opts", "hr_cg_workspace_bytes", "hr_cg_solve", "hr_force",
    "hr_link_grad", "hr_norm2", "hr_axpy", "hr_gamma5", "hr_norm2_noalloc", "hr_autotune_hop",
    "hr_tune_lookup", "hr_cg_batch_workspace_bytes", "hr_cg_solve_batch", "hr_solve_full_workspace_bytes",
    "hr_solve_full", "hr_clover_packed_bytes", "hr_clover_build", "hr_clover_apply", "hr_dirac_apply_clover",
    "hr_dirac_eo_clover", "hr_cg_clover_workspace_bytes", "hr_cg_solve_clover",
    "hr_solve_full_clover_workspace_bytes", "hr_solve_full_clover", "hr_gauge_force", "hr_gauge_action",
    "hr_link_update", "hr_mom_update", "hr_kinetic_energy", "hr_hmc_workspace_bytes", "hr_hmc_trajectory",
    "hr_clover_force_workspace_bytes", "hr_clover_insertion_force", "hr_clover_fermion_force", "hr_clover_logdet",
    "hr_ctx_status", "hr_dot", "hr_fermion_force_workspace_bytes", "hr_fermion_force", "hr_fermion_link_grad",
    "hr_fp32_fma_rate", "hr_dd_face_bytes", "hr_dd_pack_faces", "hr_dd_hop_boundary",
]


class HrError(RuntimeError):
    def __init__(self, code: int, message: str):
        self.code = code
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {message}")


class hr_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("bc", ctypes.c_int), ("theta", ctypes.c_double * 4)]


class Lattice(tuple):
    """Extents (T, L1, L2, L3) with fermion boundary conditions: ``bc`` bit mu
    makes direction mu antiperiodic; ``theta[mu]`` twists it,
    psi(x + L_mu mu) = e^{i theta_mu} psi(x) (None: no twist).  A tuple, so it
    serves wherever extents do; every call of this module that takes ``dims``
    reads ``bc`` and ``theta`` from it."""

    def __new__(cls, dims, bc: int = 0, theta=None):
        self = super().__new__(cls, (int(d) for d in dims))
        if len(self) != 4:
            raise ValueError("four extents")
        self.bc = int(bc)
        if theta is not None:
            theta = tuple(float(t) for t in theta)
            if len(theta) != 4:
                raise ValueError("four twist angles")
            if not any(theta):
                theta = None
        self.theta = theta
        return self

    def __repr__(self):
        tw = f", theta={self.theta}" if self.theta is not None else ""
        return f"Lattice({tuple(self)}, bc={self.bc}{tw})"


class hr_solver_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("inner_prec", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("n_rhs", ctypes.c_int),
                ("x0_is_guess", ctypes.c_int), ("check_every", ctypes.c_int)]


class hr_hmc_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("m0", ctypes.c_double), ("fermions", ctypes.c_int),
                ("n_steps", ctypes.c_int), ("tau", ctypes.c_double), ("integrator", ctypes.c_int),
                ("solver", hr_solver_opts), ("hasenbusch", ctypes.c_int), ("m0_hasenbusch", ctypes.c_double),
                ("n_steps_gauge", ctypes.c_int), ("clover", ctypes.c_int), ("c_sw", ctypes.c_double),
                ("clover_kind", ctypes.c_int)]


class hr_hmc_info(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("kinetic_start", ctypes.c_double), ("kinetic_end", ctypes.c_double),
                ("gauge_action_start", ctypes.c_double), ("gauge_action_end", ctypes.c_double),
                ("fermion_action_start", ctypes.c_double), ("fermion_action_end", ctypes.c_double),
                ("plaquette", ctypes.c_double), ("cg_iters", ctypes.c_int), ("solves", ctypes.c_int),
                ("seconds", ctypes.c_double)]


class hr_tune_result(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("block", ctypes.c_int), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("candidates", ctypes.c_int)]


class hr_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("n_reliable_updates", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
            LAT = hr_lattice
            sig = {
                "hr_ctx_create": ([ctypes.POINTER(P), I], I),
                "hr_ctx_destroy": ([P], I),
                "hr_last_error": ([P], ctypes.c_char_p),
                "hr_ctx_status": ([P, P], I),
                "hr_version": ([], ctypes.c_char_p),
                "hr_kappa_to_m0": ([D], D),
                "hr_m0_to_kappa": ([D], D),
                "hr_gauge_packed_bytes": ([LAT, I, I], S),
                "hr_spinor_packed_bytes": ([LAT, I, I, I, I], S),
                "hr_gauge_pack": ([P, LAT, I, I, P, P, P], I),
                "hr_spinor_pack": ([P, LAT, I, I, I, I, P, P, P], I),
                "hr_spinor_unpack": ([P, LAT, I, I, I, I, P, P, P], I),
                "hr_dirac_workspace_bytes": ([LAT, I, I, I, I], S),
                "hr_dirac_apply": ([P, LAT, D, I, I, P, P, P, P], I),
                "hr_dirac_eo": ([P, LAT, D, I, I, I, I, I, P, P, P, P, S, P], I),
                "hr_solver_default_opts": ([], hr_solver_opts),
                "hr_cg_workspace_bytes": ([LAT, I, ctypes.POINTER(hr_solver_opts)], S),
                "hr_cg_solve": ([P, LAT, D, I, ctypes.POINTER(hr_solver_opts), P, P, P,
                                 ctypes.POINTER(hr_solve_info), P, S, P], I),
                "hr_force": ([P, LAT, P, P, P, D, P, P], I),
                "hr_link_grad": ([P, LAT, P, P, D, P, P], I),
                "hr_fermion_force_workspace_bytes": ([LAT], S),
                "hr_fermion_force": ([P, LAT, D, I, P, P, P, D, P, P, S, P], I),
                "hr_fermion_link_grad": ([P, LAT, D, I, P, P, P, D, P, P, S, P], I),
                "hr_dot": ([P, LAT, I, P, P, ctypes.POINTER(D), ctypes.POINTER(D), P], I),
                "hr_fp32_fma_rate": ([P, ctypes.POINTER(D), ctypes.POINTER(D), P], I),
                "hr_dd_face_bytes": ([LAT, I, I], S),
                "hr_dd_pack_faces": ([P, LAT, I, I, I, P, P, P, P, P], I),
                "hr_dd_hop_boundary": ([P, LAT, I, I, I, P, P, P, P, P, P], I),
                "hr_norm2": ([P, LAT, I, P, ctypes.POINTER(D), P], I),
                "hr_axpy": ([P, LAT, I, D, P, P, P], I),
                "hr_gamma5": ([P, LAT, I, P, P], I),
                "hr_norm2_noalloc": ([LAT, I, I, P, P, P], I),
                "hr_cg_batch_workspace_bytes": ([I, ctypes.POINTER(LAT), I], S),
                "hr_cg_solve_batch": ([P, I, ctypes.POINTER(LAT), D, I, ctypes.POINTER(hr_solver_opts),
                                       ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                       ctypes.POINTER(hr_solve_info), P, S, P], I),
                "hr_autotune_hop": ([P, LAT, I, I, I, I, P, P, P, I, ctypes.POINTER(hr_tune_result), P], I),
                "hr_tune_lookup": ([P, LAT, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
                "hr_solve_full_workspace_bytes": ([LAT, I, ctypes.POINTER(hr_solver_opts), I], S),
                "hr_solve_full": ([P, LAT, D, I, ctypes.POINTER(hr_solver_opts), I, P, P, P,
                                   ctypes.POINTER(hr_solve_info), P, S, P], I),
                "hr_clover_packed_bytes": ([LAT, I, I], S),
                "hr_clover_build": ([P, LAT, I, I, I, D, D, P, P, P], I),
                "hr_clover_force_workspace_bytes": ([LAT], S),
                "hr_clover_insertion_force": ([P, LAT, D, P, P, D, P, P, S, P], I),
                "hr_clover_fermion_force": ([P, LAT, I, D, D, P, P, P, P, P, I, D, P, P, S, P], I),
                "hr_clover_logdet": ([P, LAT, I, P, I, ctypes.POINTER(ctypes.c_double), P], I),
                "hr_clover_apply": ([P, LAT, I, I, I, I, I, P, P, P, P], I),
                "hr_dirac_apply_clover": ([P, LAT, I, I, P, P, P, P, P], I),
                "hr_dirac_eo_clover": ([P, LAT, I, I, I, I, I, P, P, P, P, P, S, P], I),
                "hr_cg_clover_workspace_bytes": ([LAT, I, ctypes.POINTER(hr_solver_opts)], S),
                "hr_cg_solve_clover": ([P, LAT, I, ctypes.POINTER(hr_solver_opts), P, P, P, P,
                                        ctypes.POINTER(hr_solve_info), P, S, P], I),
                "hr_solve_full_clover_workspace_bytes": ([LAT, I, ctypes.POINTER(hr_solver_opts), I], S),
                "hr_solve_full_clover": ([P, LAT, I, ctypes.POINTER(hr_solver_opts), I, P, P, P, P,
                                          ctypes.POINTER(hr_solve_info), P, S, P], I),
                "hr_gauge_force": ([P, LAT, D, P, D, P, P], I),
                "hr_gauge_action": ([P, LAT, D, P, ctypes.POINTER(D), P], I),
                "hr_link_update": ([P, LAT, D, P, P, P], I),
                "hr_mom_update": ([P, LAT, D, P, P, P], I),
                "hr_kinetic_energy": ([P, LAT, P, ctypes.POINTER(D), P], I),
                "hr_hmc_workspace_bytes": ([LAT, ctypes.POINTER(hr_hmc_params)], S),
                "hr_hmc_trajectory": ([P, LAT, ctypes.POINTER(hr_hmc_params), P, P, P, P,
                                       ctypes.POINTER(hr_hmc_info), P, S, P], I),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB_PATH


# ------------------------------------------------------------------ helpers

def lattice(dims) -> hr_lattice:
    lat = hr_lattice()
    for k in range(4):
        lat.dims[k] = int(dims[k])
    lat.bc = int(getattr(dims, "bc", 0))
    theta = getattr(dims, "theta", None)
    if theta is not None:
        for k in range(4):
            lat.theta[k] = float(theta[k])
    return lat


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _nbytes(t) -> int:
    return 0 if t is None else t.numel() * t.element_size()


def _need(t, nbytes: int, what: str):
    """Buffer checks the C ABI cannot do: device residency and size."""
    if t is None or not hasattr(t, "data_ptr"):
        return
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError(f"{what}: {have} bytes given, {nbytes} needed")


class Context:
    """Owns an ``hr_ctx`` (device scratch for reductions and solver scalars)."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        rc = lib().hr_ctx_create(ctypes.byref(self._h), int(device))
        if rc != HR_OK:
            raise HrError(rc, f"hr_ctx_create(device={device}) failed")
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().hr_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        msg = lib().hr_last_error(self._h)
        return msg.decode() if msg else ""

    def check(self, rc: int):
        if rc != HR_OK:
            msg = lib().hr_last_error(self._h)
            raise HrError(rc, msg.decode() if msg else "")
        return rc


# ------------------------------------------------------------------ C entry points

def hr_ctx_status(ctx: Context, stream=None):
    """Range status of the fields packed since the last check (synchronises the
    stream); raises :class:`HrError` (HR_ERR_NUMERIC / HR_ERR_UNSUPPORTED) if a
    packed value was non-finite or above 2^120 in magnitude."""
    ctx.check(lib().hr_ctx_status(ctx.handle, _stream(stream)))


def hr_version() -> str:
    return lib().hr_version().decode()


def hr_kappa_to_m0(kappa: float) -> float:
    return lib().hr_kappa_to_m0(float(kappa))


def hr_m0_to_kappa(m0: float) -> float:
    return lib().hr_m0_to_kappa(float(m0))


def hr_gauge_packed_bytes(dims, rep: int, prec: int) -> int:
    return int(lib().hr_gauge_packed_bytes(lattice(dims), rep, prec))


def hr_spinor_packed_bytes(dims, rep: int, prec: int, parity: int, n_rhs: int = 1) -> int:
    return int(lib().hr_spinor_packed_bytes(lattice(dims), rep, prec, parity, n_rhs))


def hr_dirac_workspace_bytes(dims, rep: int, prec: int, op: int, n_rhs: int = 1) -> int:
    return int(lib().hr_dirac_workspace_bytes(lattice(dims), rep, prec, op, n_rhs))


def hr_gauge_pack(ctx: Context, dims, rep, prec, canonical, packed, stream=None):
    V = _vol(dims)
    _need(canonical, 4 * V * 4 * 8, "canonical gauge")
    _need(packed, hr_gauge_packed_bytes(dims, rep, prec), "packed gauge")
    return ctx.check(lib().hr_gauge_pack(ctx.handle, lattice(dims), rep, prec, _ptr(canonical),
                                         _ptr(packed), _stream(stream)))


def hr_spinor_pack(ctx: Context, dims, rep, prec, parity, n_rhs, canonical, packed, stream=None):
    nc = 2 if rep == HR_FUND else 3
    _need(canonical, n_rhs * _vol(dims) * 4 * nc * 16, "canonical spinor")
    _need(packed, hr_spinor_packed_bytes(dims, rep, prec, parity, n_rhs), "packed spinor")
    return ctx.check(lib().hr_spinor_pack(ctx.handle, lattice(dims), rep, prec, parity, n_rhs,
                                          _ptr(canonical), _ptr(packed), _stream(stream)))


def hr_spinor_unpack(ctx: Context, dims, rep, prec, parity, n_rhs, packed, canonical, stream=None):
    nc = 2 if rep == HR_FUND else 3
    _need(canonical, n_rhs * _vol(dims) * 4 * nc * 16, "canonical spinor")
    _need(packed, hr_spinor_packed_bytes(dims, rep, prec, parity, n_rhs), "packed spinor")
    return ctx.check(lib().hr_spinor_unpack(ctx.handle, lattice(dims), rep, prec, parity, n_rhs,
                                            _ptr(packed), _ptr(canonical), _stream(stream)))


def hr_dirac_apply(ctx: Context, dims, m0, rep, prec, gauge, inp, out, stream=None):
    full = hr_spinor_packed_bytes(dims, rep, prec, HR_FULL, 1)
    _need(inp, full, "in")
    _need(out, full, "out")
    return ctx.check(lib().hr_dirac_apply(ctx.handle, lattice(dims), float(m0), rep, prec,
                                          _ptr(gauge), _ptr(inp), _ptr(out), _stream(stream)))


def hr_dirac_eo(ctx: Context, dims, m0, rep, prec, out_parity, op, n_rhs, gauge, inp, out,
                work=None, stream=None):
    half = hr_spinor_packed_bytes(dims, rep, prec, HR_EVEN, n_rhs)
    _need(inp, half, "in")
    _need(out, half, "out")
    wb = 0 if work is None else work.numel() * work.element_size()
    return ctx.check(lib().hr_dirac_eo(ctx.handle, lattice(dims), float(m0), rep, prec, out_parity,
                                       op, n_rhs, _ptr(gauge), _ptr(inp), _ptr(out), _ptr(work),
                                       wb, _stream(stream)))


def hr_solver_default_opts() -> hr_solver_opts:
    return lib().hr_solver_default_opts()


def hr_cg_workspace_bytes(dims, rep: int, opts: hr_solver_opts) -> int:
    return int(lib().hr_cg_workspace_bytes(lattice(dims), rep, ctypes.byref(opts)))


def hr_cg_solve(ctx: Context, dims, m0, rep, opts: hr_solver_opts, gauge, b, x, work, stream=None,
                raise_on_error: bool = True):
    """Returns (status, hr_solve_info)."""
    half = hr_spinor_packed_bytes(dims, rep, HR_F64, HR_EVEN, opts.n_rhs)
    _need(b, half, "b")
    _need(x, half, "x")
    info = hr_solve_info()
    wb = 0 if work is None else work.numel() * work.element_size()
    rc = lib().hr_cg_solve(ctx.handle, lattice(dims), float(m0), rep, ctypes.byref(opts),
                           _ptr(gauge), _ptr(b), _ptr(x), ctypes.byref(info), _ptr(work), wb,
                           _stream(stream))
    if raise_on_error and rc not in (HR_OK, HR_ERR_NOT_CONVERGED):
        ctx.check(rc)
    return rc, info


def hr_solve_full_workspace_bytes(dims, rep, opts: hr_solver_opts, system: int) -> int:
    return int(lib().hr_solve_full_workspace_bytes(lattice(dims), rep, ctypes.byref(opts), system))


def hr_solve_full(ctx: Context, dims, m0, rep, opts: hr_solver_opts, system, gauge, b, x, work, stream=None,
                  raise_on_error: bool = True):
    """D x = b (HR_SYSTEM_D) or D^+ D x = b (HR_SYSTEM_DDAG_D) on full packed
    FP64 spinors.  Returns (status, hr_solve_info)."""
    full = hr_spinor_packed_bytes(dims, rep, HR_F64, HR_FULL, 1)
    _need(b, full, "b")
    _need(x, full, "x")
    info = hr_solve_info()
    wb = 0 if work is None else work.numel() * work.element_size()
    rc = lib().hr_solve_full(ctx.handle, lattice(dims), float(m0), rep, ctypes.byref(opts), int(system),
                             _ptr(gauge), _ptr(b), _ptr(x), ctypes.byref(info), _ptr(work), wb,
                             _stream(stream))
    if raise_on_error and rc not in (HR_OK, HR_ERR_NOT_CONVERGED):
        ctx.check(rc)
    return rc, info


# ---- clover and exponential-clover site terms

def hr_clover_packed_bytes(dims, rep: int, prec: int) -> int:
    return int(lib().hr_clover_packed_bytes(lattice(dims), rep, prec))


def hr_clover_build(ctx: Context, dims, rep, prec, kind, m0, c_sw, canonical, clover, stream=None):
    """Packed clover field (A and A^-1 on both parities) from the canonical gauge."""
    _need(canonical, 4 * _vol(dims) * 4 * 8, "canonical gauge")
    _need(clover, hr_clover_packed_bytes(dims, rep, prec), "clover")
    return ctx.check(lib().hr_clover_build(ctx.handle, lattice(dims), rep, prec, int(kind), float(m0), float(c_sw),
                                           _ptr(canonical), _ptr(clover), _stream(stream)))


def hr_clover_force_workspace_bytes(dims) -> int:
    return int(lib().hr_clover_force_workspace_bytes(lattice(dims)))


def hr_clover_insertion_force(ctx: Context, dims, c_sw, gauge, lam, coeff, force, work, stream=None):
    """force += coeff c_sw d/dw Re sum tr[C lam]; lam complex128 [V, 8, 8] on the device."""
    V = _vol(dims)
    _need(gauge, 4 * V * 4 * 8, "gauge")
    _need(lam, V * 64 * 16, "lam")
    _need(force, 4 * V * 3 * 8, "force")
    return ctx.check(lib().hr_clover_insertion_force(ctx.handle, lattice(dims), float(c_sw), _ptr(gauge), _ptr(lam),
                                                     float(coeff), _ptr(force), _ptr(work), _nbytes(work),
                                                     _stream(stream)))


def hr_clover_fermion_force(ctx: Context, dims, m0, c_sw, gauge, gauge_packed, clover, X, with_det, coeff, force,
                            work, stream=None, kind=HR_CLOVER_SW, Y=None):
    V = _vol(dims)
    _need(gauge, 4 * V * 4 * 8, "gauge")
    _need(force, 4 * V * 3 * 8, "force")
    _need(X, hr_spinor_packed_bytes(dims, HR_FUND, HR_F64, HR_EVEN, 1), "X")
    return ctx.check(lib().hr_clover_fermion_force(ctx.handle, lattice(dims), int(kind), float(m0), float(c_sw),
                                                   _ptr(gauge),
                                                   _ptr(gauge_packed), _ptr(clover), _ptr(X), _ptr(Y),
                                                   int(bool(with_det)),
                                                   float(coeff), _ptr(force), _ptr(work), _nbytes(work),
                                                   _stream(stream)))


def hr_clover_logdet(ctx: Context, dims, rep, clover, parity, stream=None) -> float:
    out = ctypes.c_double(0.0)
    ctx.check(lib().hr_clover_logdet(ctx.handle, lattice(dims), rep, _ptr(clover), parity, ctypes.byref(out),
                                     _stream(stream)))
    return out.value


def hr_clover_apply(ctx: Context, dims, rep, prec, parity, inverse, n_rhs, clover, inp, out, stream=None):
    half = hr_spinor_packed_bytes(dims, rep, prec, parity, n_rhs)
    _need(inp, half, "in")
    _need(out, half, "out")
    return ctx.check(lib().hr_clover_apply(ctx.handle, lattice(dims), rep, prec, parity, int(bool(inverse)), n_rhs,
                                           _ptr(clover), _ptr(inp), _ptr(out), _stream(stream)))


def hr_dirac_apply_clover(ctx: Context, dims, rep, prec, gauge, clover, inp, out, stream=None):
    full = hr_spinor_packed_bytes(dims, rep, prec, HR_FULL, 1)
    _need(inp, full, "in")
    _need(out, full, "out")
    return ctx.check(lib().hr_dirac_apply_clover(ctx.handle, lattice(dims), rep, prec, _ptr(gauge), _ptr(clover),
                                                 _ptr(inp), _ptr(out), _stream(stream)))


def hr_dirac_eo_clover(ctx: Context, dims, rep, prec, out_parity, op, n_rhs, gauge, clover, inp, out,
                       work=None, stream=None):
    half = hr_spinor_packed_bytes(dims, rep, prec, HR_EVEN, n_rhs)
    _need(inp, half, "in")
    _need(out, half, "out")
    wb = 0 if work is None else work.numel() * work.element_size()
    return ctx.check(lib().hr_dirac_eo_clover(ctx.handle, lattice(dims), rep, prec, out_parity, op, n_rhs,
                                              _ptr(gauge), _ptr(clover), _ptr(inp), _ptr(out), _ptr(work), wb,
                                              _stream(stream)))


def hr_cg_clover_workspace_bytes(dims, rep: int, opts: hr_solver_opts) -> int:
    return int(lib().hr_cg_clover_workspace_bytes(lattice(dims), rep, ctypes.byref(opts)))


def hr_cg_solve_clover(ctx: Context, dims, rep, opts: hr_solver_opts, gauge, clover, b, x, work, stream=None,
                       raise_on_error: bool = True):
    """CG on Mhat^+ Mhat with the clover site term.  Returns (status, hr_solve_info)."""
    half = hr_spinor_packed_bytes(dims, rep, HR_F64, HR_EVEN, opts.n_rhs)
    _need(b, half, "b")
    _need(x, half, "x")
    info = hr_solve_info()
    wb = 0 if work is None else work.numel() * work.element_size()
    rc = lib().hr_cg_solve_clover(ctx.handle, lattice(dims), rep, ctypes.byref(opts), _ptr(gauge), _ptr(clover),
                                  _ptr(b), _ptr(x), ctypes.byref(info), _ptr(work), wb, _stream(stream))
    if raise_on_error and rc not in (HR_OK, HR_ERR_NOT_CONVERGED):
        ctx.check(rc)
    return rc, info


def hr_solve_full_clover_workspace_bytes(dims, rep, opts: hr_solver_opts, system: int) -> int:
    return int(lib().hr_solve_full_clover_workspace_bytes(lattice(dims), rep, ctypes.byref(opts), system))


def hr_solve_full_clover(ctx: Context, dims, rep, opts: hr_solver_opts, system, gauge, clover, b, x, work,
                         stream=None, raise_on_error: bool = True):
    """D x = b or D^+ D x = b with the clover site term.  Returns (status, hr_solve_info)."""
    full = hr_spinor_packed_bytes(dims, rep, HR_F64, HR_FULL, 1)
    _need(b, full, "b")
    _need(x, full, "x")
    info = hr_solve_info()
    wb = 0 if work is None else work.numel() * work.element_size()
    rc = lib().hr_solve_full_clover(ctx.handle, lattice(dims), rep, ctypes.byref(opts), int(system), _ptr(gauge),
                                    _ptr(clover), _ptr(b), _ptr(x), ctypes.byref(info), _ptr(work), wb,
                                    _stream(stream))
    if raise_on_error and rc not in (HR_OK, HR_ERR_NOT_CONVERGED):
        ctx.check(rc)
    return rc, info


# ---- HMC molecular dynamics

def _links(dims):
    return 4 * _vol(dims)


def hr_gauge_force(ctx: Context, dims, beta, gauge, coeff, force, stream=None):
    _need(gauge, _links(dims) * 4 * 8, "gauge")
    _need(force, _links(dims) * 3 * 8, "force")
    return ctx.check(lib().hr_gauge_force(ctx.handle, lattice(dims), float(beta), _ptr(gauge), float(coeff),
                                          _ptr(force), _stream(stream)))


def hr_gauge_action(ctx: Context, dims, beta, gauge, stream=None) -> float:
    _need(gauge, _links(dims) * 4 * 8, "gauge")
    out = ctypes.c_double(0.0)
    ctx.check(lib().hr_gauge_action(ctx.handle, lattice(dims), float(beta), _ptr(gauge), ctypes.byref(out),
                                    _stream(stream)))
    return out.value


def hr_link_update(ctx: Context, dims, eps, mom, gauge, stream=None):
    _need(mom, _links(dims) * 3 * 8, "mom")
    _need(gauge, _links(dims) * 4 * 8, "gauge")
    return ctx.check(lib().hr_link_update(ctx.handle, lattice(dims), float(eps), _ptr(mom), _ptr(gauge),
                                          _stream(stream)))


def hr_mom_update(ctx: Context, dims, eps, force, mom, stream=None):
    _need(force, _links(dims) * 3 * 8, "force")
    _need(mom, _links(dims) * 3 * 8, "mom")
    return ctx.check(lib().hr_mom_update(ctx.handle, lattice(dims), float(eps), _ptr(force), _ptr(mom),
                                         _stream(stream)))


def hr_kinetic_energy(ctx: Context, dims, mom, stream=None) -> float:
    _need(mom, _links(dims) * 3 * 8, "mom")
    out = ctypes.c_double(0.0)
    ctx.check(lib().hr_kinetic_energy(ctx.handle, lattice(dims), _ptr(mom), ctypes.byref(out), _stream(stream)))
    return out.value


def hr_hmc_params_default(beta: float, m0: float = 0.0, fermions: bool = True, n_steps: int = 10,
                          tau: float = 1.0, integrator: int = HR_INTEGRATOR_OMELYAN) -> hr_hmc_params:
    prm = hr_hmc_params()
    prm.beta, prm.m0, prm.fermions = float(beta), float(m0), int(bool(fermions))
    prm.n_steps, prm.tau, prm.integrator = int(n_steps), float(tau), int(integrator)
    prm.solver = hr_solver_default_opts()
    prm.n_steps_gauge = 1
    return prm


def hr_hmc_workspace_bytes(dims, prm: hr_hmc_params) -> int:
    return int(lib().hr_hmc_workspace_bytes(lattice(dims), ctypes.byref(prm)))


def hr_hmc_trajectory(ctx: Context, dims, prm: hr_hmc_params, gauge, mom, eta, work, stream=None, phi=None):
    """One MD trajectory, gauge and mom updated in place (phi: the Hasenbusch
    ratio pseudofermion when prm.hasenbusch).  Returns hr_hmc_info."""
    _need(gauge, _links(dims) * 4 * 8, "gauge")
    _need(mom, _links(dims) * 3 * 8, "mom")
    half = hr_spinor_packed_bytes(dims, HR_FUND, HR_F64, HR_EVEN, 1)
    if prm.fermions:
        _need(eta, half, "eta")
    if prm.hasenbusch:
        _need(phi, half, "phi")
    info = hr_hmc_info()
    wb = 0 if work is None else work.numel() * work.element_size()
    ctx.check(lib().hr_hmc_trajectory(ctx.handle, lattice(dims), ctypes.byref(prm), _ptr(gauge), _ptr(mom),
                                      _ptr(eta), _ptr(phi), ctypes.byref(info), _ptr(work), wb, _stream(stream)))
    return info


def hr_force(ctx: Context, dims, gauge, a_full, b_full, beta, force, stream=None):
    _need(force, 4 * _vol(dims) * 3 * 8, "force")
    return ctx.check(lib().hr_force(ctx.handle, lattice(dims), _ptr(gauge), _ptr(a_full),
                                    _ptr(b_full), float(beta), _ptr(force), _stream(stream)))


def hr_link_grad(ctx: Context, dims, a_full, b_full, beta, grad, stream=None):
    _need(grad, 4 * _vol(dims) * 4 * 8, "grad")
    return ctx.check(lib().hr_link_grad(ctx.handle, lattice(dims), _ptr(a_full), _ptr(b_full),
                                        float(beta), _ptr(grad), _stream(stream)))


def hr_fermion_force_workspace_bytes(dims) -> int:
    return int(lib().hr_fermion_force_workspace_bytes(lattice(dims)))


def hr_fermion_force(ctx: Context, dims, m0, rep, gauge, X, L, coeff, force, work, stream=None):
    """force += coeff d/dw Re<L, Mhat^+ Mhat X> (L = None: L = X)."""
    _need(force, 4 * _vol(dims) * 3 * 8, "force")
    return ctx.check(lib().hr_fermion_force(ctx.handle, lattice(dims), float(m0), rep, _ptr(gauge), _ptr(X),
                                            _ptr(L), float(coeff), _ptr(force), _ptr(work), _nbytes(work),
                                            _stream(stream)))


def hr_fermion_link_grad(ctx: Context, dims, m0, rep, gauge, X, L, coeff, grad, work, stream=None):
    """grad += coeff d/dq Re<L, Mhat^+ Mhat X> (L = None: L = X)."""
    _need(grad, 4 * _vol(dims) * 4 * 8, "grad")
    return ctx.check(lib().hr_fermion_link_grad(ctx.handle, lattice(dims), float(m0), rep, _ptr(gauge), _ptr(X),
                                                _ptr(L), float(coeff), _ptr(grad), _ptr(work), _nbytes(work),
                                                _stream(stream)))


def hr_dot(ctx: Context, dims, rep, a, b, stream=None) -> complex:
    """<a, b> = sum conj(a) b over packed FP64 fields of one parity."""
    re, im = ctypes.c_double(0.0), ctypes.c_double(0.0)
    ctx.check(lib().hr_dot(ctx.handle, lattice(dims), rep, _ptr(a), _ptr(b), ctypes.byref(re), ctypes.byref(im),
                           _stream(stream)))
    return complex(re.value, im.value)


def hr_fp32_fma_rate(ctx: Context, stream=None):
    """Measured FP32 FMA pipe rate (scalar, packed f32x2) in lane operations per second."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    ctx.check(lib().hr_fp32_fma_rate(ctx.handle, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return a.value, b.value


def hr_dd_face_bytes(local_dims, rep, prec) -> int:
    return int(lib().hr_dd_face_bytes(lattice(local_dims), rep, prec))


def hr_dd_pack_faces(ctx: Context, local_dims, rep, prec, in_parity, gauge, inp, to_lower, to_upper, stream=None):
    return ctx.check(lib().hr_dd_pack_faces(ctx.handle, lattice(local_dims), rep, prec, in_parity, _ptr(gauge),
                                            _ptr(inp), _ptr(to_lower), _ptr(to_upper), _stream(stream)))


def hr_dd_hop_boundary(ctx: Context, local_dims, rep, prec, out_parity, gauge, inp, from_lower, from_upper, out,
                       stream=None):
    return ctx.check(lib().hr_dd_hop_boundary(ctx.handle, lattice(local_dims), rep, prec, out_parity, _ptr(gauge),
                                              _ptr(inp), _ptr(from_lower), _ptr(from_upper), _ptr(out),
                                              _stream(stream)))


def hr_norm2(ctx: Context, dims, rep, v, stream=None) -> float:
    out = ctypes.c_double(0.0)
    ctx.check(lib().hr_norm2(ctx.handle, lattice(dims), rep, _ptr(v), ctypes.byref(out),
                             _stream(stream)))
    return out.value


def hr_axpy(ctx: Context, dims, rep, a, x, y, stream=None):
    return ctx.check(lib().hr_axpy(ctx.handle, lattice(dims), rep, float(a), _ptr(x), _ptr(y),
                                   _stream(stream)))


def hr_gamma5(ctx: Context, dims, rep, v, stream=None):
    return ctx.check(lib().hr_gamma5(ctx.handle, lattice(dims), rep, _ptr(v), _stream(stream)))


def _vol(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def hr_norm2_noalloc(dims, rep, n_rhs, v, result, stream=None) -> int:
    """|v_r|^2 into the device tensor ``result`` without a context or any
    allocation (for callers that may not allocate device memory).  Returns the
    library's status code; raises ValueError only when ``result`` is not a
    contiguous CUDA tensor of at least n_rhs doubles."""
    _need(result, 8 * int(n_rhs), "result")
    return int(lib().hr_norm2_noalloc(lattice(dims), rep, int(n_rhs), _ptr(v), _ptr(result),
                                      _stream(stream)))


def hr_autotune_hop(ctx: Context, dims, rep, prec, out_parity, n_rhs, gauge, inp, out, reps=20,
                    stream=None) -> hr_tune_result:
    half = hr_spinor_packed_bytes(dims, rep, prec, HR_EVEN, n_rhs)
    _need(inp, half, "in")
    _need(out, half, "out")
    res = hr_tune_result()
    ctx.check(lib().hr_autotune_hop(ctx.handle, lattice(dims), rep, prec, out_parity, n_rhs, _ptr(gauge),
                                    _ptr(inp), _ptr(out), int(reps), ctypes.byref(res), _stream(stream)))
    return res


def hr_tune_lookup(ctx: Context, dims, rep, prec, n_rhs=1):
    v, b = ctypes.c_int(-1), ctypes.c_int(-1)
    ctx.check(lib().hr_tune_lookup(ctx.handle, lattice(dims), rep, prec, n_rhs, ctypes.byref(v),
                                   ctypes.byref(b)))
    return v.value, b.value


def _lattice_array(dims_list):
    arr = (hr_lattice * len(dims_list))()
    for k, d in enumerate(dims_list):
        arr[k] = lattice(d)
    return arr


def hr_cg_batch_workspace_bytes(dims_list, rep) -> int:
    return int(lib().hr_cg_batch_workspace_bytes(len(dims_list), _lattice_array(dims_list), rep))


def hr_cg_solve_batch(ctx: Context, dims_list, m0, rep, opts: hr_solver_opts, gauges, bs, xs, work,
                      stream=None, raise_on_error: bool = True):
    """Batched solve of len(dims_list) lattices; returns (status, [hr_solve_info])."""
    n = len(dims_list)
    for k, d in enumerate(dims_list):
        half = hr_spinor_packed_bytes(d, rep, HR_F64, HR_EVEN, 1)
        _need(bs[k], half, f"b[{k}]")
        _need(xs[k], half, f"x[{k}]")
    P = ctypes.c_void_p
    garr = (P * n)(*[_ptr(g) for g in gauges])
    barr = (P * n)(*[_ptr(b) for b in bs])
    xarr = (P * n)(*[_ptr(x) for x in xs])
    infos = (hr_solve_info * n)()
    wb = 0 if work is None else work.numel() * work.element_size()
    rc = lib().hr_cg_solve_batch(ctx.handle, n, _lattice_array(dims_list), float(m0), rep, ctypes.byref(opts),
                                 garr, barr, xarr, infos, _ptr(work), wb, _stream(stream))
    if raise_on_error and rc not in (HR_OK, HR_ERR_NOT_CONVERGED):
        ctx.check(rc)
    return rc, list(infos)
