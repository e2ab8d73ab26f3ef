"""torch.autograd.Function wrappers of the Dirac operator and of the even-odd
solve, with hand-written backward passes that run in the library's kernels.

Conventions: links ``q`` are the canonical quaternion field, float64
``[4, V, 4]``; spinors are complex128 ``[V, 4, 2]`` (fundamental).  For a real
loss L and a complex tensor z, torch's gradient is dL/dRe z + i dL/dIm z, so
for y = A z with A linear, grad_z = A^+ grad_y.

* :class:`DiracApply` -- y = D(U) psi on the full lattice.
  backward: grad_psi = D^+ g = g5 D g5 g (gamma5-hermiticity), and
  grad_q[mu, x, k] = -1/2 d Re<g, H psi> / d q_k (``hr_link_grad``).
* :class:`EoSolve` -- x = (Mhat^+ Mhat)^-1 eta on even sites (eta and x are
  full-lattice tensors whose odd sites are zero).  backward: one extra solve
  lambda = A^-1 grad_x (A is Hermitian), grad_eta = lambda, and
  grad_q = -d Re<lambda, A x> / dq at fixed x, lambda (``hr_fermion_link_grad``).
* :func:`fermion_force` -- the su(2) force of S = Re<eta, (Mhat^+ Mhat)^-1 eta>,
  -d Re<x, A x> / dw at x = A^-1 eta (``hr_fermion_force``), and S = Re<eta, x>
  (``hr_dot``).

These are the differentiable solve and the fermion force of the HMC that
consumes the even-odd preconditioned operator (arXiv:2411.18511, Sec. 2.1).
Byte copies between packed buffers are plain device memory moves; every
arithmetic step runs in libhirep_gb300's kernels.
"""

from __future__ import annotations

import threading

import torch

from . import fields, hr

_ctx_lock = threading.Lock()
_contexts: dict[int, hr.Context] = {}


def default_context(device: int | None = None) -> hr.Context:
    """One library context per CUDA device, created on first use."""
    dev = torch.cuda.current_device() if device is None else int(device)
    with _ctx_lock:
        if dev not in _contexts:
            _contexts[dev] = hr.Context(dev)
        return _contexts[dev]


def _check_dims(q: torch.Tensor, dims):
    V = 1
    for d in dims:
        V *= int(d)
    if tuple(q.shape) != (4, V, 4):
        raise ValueError(f"links must have shape (4, {V}, 4), got {tuple(q.shape)}")
    return hr.Lattice(dims, getattr(dims, "bc", 0), getattr(dims, "theta", None))  # keeps the boundary conditions


class _Lattice:
    """Packed FP64 fundamental fields of one lattice and the kernels on them."""

    def __init__(self, dims, q: torch.Tensor):
        self.ctx = default_context(q.device.index)
        self.dims = dims
        self.dev = q.device
        self.gauge = fields.pack_gauge(self.ctx, dims, hr.HR_FUND, hr.HR_F64, q.detach().contiguous())
        self.half = hr.hr_spinor_packed_bytes(dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, 1)

    # packed buffers: a full field is [even half | odd half]
    def full(self, psi=None) -> torch.Tensor:
        if psi is None:
            return torch.zeros(2 * self.half, dtype=torch.uint8, device=self.dev)
        return fields.pack_spinor(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, psi.detach().contiguous())

    def even(self, psi=None) -> torch.Tensor:
        if psi is None:
            return torch.zeros(self.half, dtype=torch.uint8, device=self.dev)
        return fields.pack_spinor(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, psi.detach().contiguous())

    def ev(self, p_full):
        return p_full[: self.half]

    def od(self, p_full):
        return p_full[self.half: 2 * self.half]

    def unpack_full(self, p):
        return fields.unpack_spinor(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, hr.HR_FULL, p)

    def unpack_even(self, p):
        return fields.unpack_spinor(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, p)

    # operators
    def dirac(self, m0, src_full, dst_full):
        hr.hr_dirac_apply(self.ctx, self.dims, m0, hr.HR_FUND, hr.HR_F64, self.gauge, src_full, dst_full)

    def gamma5(self, p_half):
        hr.hr_gamma5(self.ctx, self.dims, hr.HR_FUND, p_half)

    def solve(self, m0, b_even, tol, maxiter):
        opts = hr.hr_solver_default_opts()
        opts.tol = tol
        opts.maxiter = maxiter
        work = fields.empty_bytes(hr.hr_cg_workspace_bytes(self.dims, hr.HR_FUND, opts), self.dev)
        x = self.even()
        rc, info = hr.hr_cg_solve(self.ctx, self.dims, m0, hr.HR_FUND, opts, self.gauge, b_even, x, work)
        if rc != hr.HR_OK:
            raise hr.HrError(rc, f"solve did not reach tol={tol}: residual {info.true_rel_residual:.3e}")
        return x, info

    def force_work(self):
        return fields.empty_bytes(hr.hr_fermion_force_workspace_bytes(self.dims), self.dev)


class DiracApply(torch.autograd.Function):
    """y = D(U) psi (full lattice, SU(2) fundamental, FP64-class arithmetic)."""

    @staticmethod
    def forward(ctx, q, psi, dims, m0):
        dims = _check_dims(q, dims)
        lat = _Lattice(dims, q)
        dst = lat.full()
        lat.dirac(m0, lat.full(psi), dst)
        ctx.save_for_backward(q, psi)
        ctx.dims, ctx.m0 = dims, m0
        return lat.unpack_full(dst)

    @staticmethod
    def backward(ctx, g):
        q, psi = ctx.saved_tensors
        lat = _Lattice(ctx.dims, q)
        gp = lat.full(g.contiguous())
        grad_q = grad_psi = None
        if ctx.needs_input_grad[1]:
            t = gp.clone()                      # D^+ g = g5 D g5 g
            lat.gamma5(lat.ev(t))
            lat.gamma5(lat.od(t))
            out = lat.full()
            lat.dirac(ctx.m0, t, out)
            lat.gamma5(lat.ev(out))
            lat.gamma5(lat.od(out))
            grad_psi = lat.unpack_full(out)
        if ctx.needs_input_grad[0]:
            grad_q = torch.zeros_like(q)
            hr.hr_link_grad(lat.ctx, ctx.dims, gp, lat.full(psi), -0.5, grad_q)
        return grad_q, grad_psi, None, None


class EoSolve(torch.autograd.Function):
    """x = (Mhat^+ Mhat)^-1 eta on even sites (odd sites of eta are ignored, of x zero)."""

    @staticmethod
    def forward(ctx, q, eta, dims, m0, tol=1e-12, maxiter=20000):
        dims = _check_dims(q, dims)
        lat = _Lattice(dims, q)
        x, info = lat.solve(m0, lat.even(eta), tol, maxiter)
        ctx.save_for_backward(q)
        ctx.x = x
        ctx.dims, ctx.m0, ctx.tol, ctx.maxiter = dims, m0, tol, maxiter
        return lat.unpack_even(x)

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        lat = _Lattice(ctx.dims, q)
        lam, _ = lat.solve(ctx.m0, lat.even(g.contiguous()), ctx.tol, ctx.maxiter)
        grad_eta = lat.unpack_even(lam) if ctx.needs_input_grad[1] else None
        grad_q = None
        if ctx.needs_input_grad[0]:
            grad_q = torch.zeros_like(q)
            hr.hr_fermion_link_grad(lat.ctx, ctx.dims, ctx.m0, hr.HR_FUND, lat.gauge, ctx.x, lam, -1.0, grad_q,
                                    lat.force_work())
        return grad_q, grad_eta, None, None, None, None


def fermion_force(q: torch.Tensor, eta: torch.Tensor, dims, m0, tol=1e-12):
    """su(2) force F[mu, x, a] = dS/dw_a of S = Re<eta, (Mhat^+ Mhat)^-1 eta> under
    U_mu(x) -> exp(i w.s/2) U_mu(x): one solve and one force kernel.  Returns (F, S)."""
    dims = _check_dims(q, dims)
    lat = _Lattice(dims, q)
    e = lat.even(eta)
    x, _ = lat.solve(m0, e, tol, 20000)
    F = torch.zeros((4, q.shape[1], 3), dtype=torch.float64, device=q.device)
    hr.hr_fermion_force(lat.ctx, dims, m0, hr.HR_FUND, lat.gauge, x, None, -1.0, F, lat.force_work())
    S = hr.hr_dot(lat.ctx, dims, hr.HR_FUND, e, x).real
    return F, torch.tensor(S, dtype=torch.float64, device=q.device)
