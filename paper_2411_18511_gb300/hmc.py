"""Hybrid Monte Carlo for SU(2) with two flavours of even-odd preconditioned
Wilson fermions (fundamental) on one GPU: the Markov chain around
``hr_hmc_trajectory`` (the molecular dynamics runs in the library's kernels).

Each step draws Gaussian momenta and a pseudofermion eta = Mhat^+ xi with
P(xi) ~ exp(-xi^+ xi), integrates one trajectory, and accepts the new links
with probability min(1, exp(-dH)); a rejected trajectory restores the links.
With clover fermions (``c_sw``) eta = Mhat^+ xi with the clover Schur
operator.  With Hasenbusch mass preconditioning (``m0_hasenbusch``) it draws two:
eta = Mhat_H^+ xi1 and phi = Mhat_H (Mhat_H^+ Mhat_H)^-1 Mhat^+ xi2 (one
solve at the heavy mass).  The random numbers come from a seeded torch
generator on the device.
"""

from __future__ import annotations

import math

import torch

from . import fields, hr


class HMC:
    def __init__(self, ctx: hr.Context, dims, beta: float, m0: float = 0.0, fermions: bool = True,
                 n_steps: int = 10, tau: float = 1.0, integrator: int = hr.HR_INTEGRATOR_OMELYAN,
                 solver: hr.hr_solver_opts | None = None, seed: int = 0, device="cuda",
                 m0_hasenbusch: float | None = None, n_steps_gauge: int = 1, c_sw: float | None = None,
                 clover_kind: int = hr.HR_CLOVER_SW):
        self.ctx, self.dims, self.device = ctx, dims, device
        self.prm = hr.hr_hmc_params_default(beta, m0, fermions, n_steps, tau, integrator)
        if solver is not None:
            self.prm.solver = solver
        if m0_hasenbusch is not None:
            self.prm.hasenbusch = 1
            self.prm.m0_hasenbusch = float(m0_hasenbusch)
        self.prm.n_steps_gauge = int(n_steps_gauge)
        if c_sw is not None:
            self.prm.clover = 1
            self.prm.c_sw = float(c_sw)
            self.prm.clover_kind = int(clover_kind)
        self.work = fields.empty_bytes(hr.hr_hmc_workspace_bytes(dims, self.prm), device)
        self.V = fields.volume(dims)
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(int(seed))
        self.accepted = 0
        self.trajectories = 0

    def draw_momenta(self) -> torch.Tensor:
        return torch.randn((4, self.V, 3), dtype=torch.float64, device=self.device, generator=self.gen)

    def _xi(self):
        """Packed even complex Gaussian field with <|xi|^2> = 1 per component."""
        shape = (self.V, 4, 2)
        xi = torch.complex(torch.randn(shape, dtype=torch.float64, device=self.device, generator=self.gen),
                           torch.randn(shape, dtype=torch.float64, device=self.device, generator=self.gen))
        return fields.pack_spinor(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, xi / math.sqrt(2.0))

    def _schur(self, gauge, m0, src, dagger, clover=None):
        d = self.dims
        op = hr.HR_OP_SCHUR_DAG if dagger else hr.HR_OP_SCHUR
        out = fields.empty_spinor(d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, device=self.device)
        work = fields.empty_bytes(hr.hr_dirac_workspace_bytes(d, hr.HR_FUND, hr.HR_F64, op), self.device)
        if clover is not None:
            hr.hr_dirac_eo_clover(self.ctx, d, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, op, 1, gauge, clover, src, out, work)
        else:
            hr.hr_dirac_eo(self.ctx, d, m0, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, op, 1, gauge, src, out, work)
        return out

    def draw_pseudofermion(self, q: torch.Tensor):
        """Packed even eta = Mhat^+ xi for the links q (Hasenbusch: eta = Mhat_H^+ xi1
        and phi = Mhat_H (Mhat_H^+ Mhat_H)^-1 Mhat^+ xi2; returns (eta, phi))."""
        gauge = fields.pack_gauge(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, q)
        m0, mh = self.prm.m0, self.prm.m0_hasenbusch
        clov = clov_h = None
        if self.prm.clover:
            def build(m):
                return fields.build_clover(self.ctx, self.dims, hr.HR_FUND, hr.HR_F64, self.prm.clover_kind, m,
                                           self.prm.c_sw, q)

            clov = build(m0)
            if self.prm.hasenbusch:
                clov_h = build(mh)
        if not self.prm.hasenbusch:
            return self._schur(gauge, m0, self._xi(), True, clov)
        eta = self._schur(gauge, mh, self._xi(), True, clov_h)
        rhs = self._schur(gauge, m0, self._xi(), True, clov)
        opts = hr.hr_solver_opts.from_buffer_copy(self.prm.solver)
        opts.tol = min(opts.tol, 1e-12)
        y = fields.zeros_spinor(self.dims, hr.HR_FUND, hr.HR_F64, hr.HR_EVEN, device=self.device)
        if clov_h is not None:
            work = fields.empty_bytes(hr.hr_cg_clover_workspace_bytes(self.dims, hr.HR_FUND, opts), self.device)
            hr.hr_cg_solve_clover(self.ctx, self.dims, hr.HR_FUND, opts, gauge, clov_h, rhs, y, work)
        else:
            work = fields.empty_bytes(hr.hr_cg_workspace_bytes(self.dims, hr.HR_FUND, opts), self.device)
            hr.hr_cg_solve(self.ctx, self.dims, mh, hr.HR_FUND, opts, gauge, rhs, y, work)
        return eta, self._schur(gauge, mh, y, False, clov_h)

    def step(self, q: torch.Tensor):
        """One HMC update of the links q (device double[4][V][4], in place).
        Returns (accepted, hr_hmc_info)."""
        backup = q.clone()
        p = self.draw_momenta()
        eta = phi = None
        if self.prm.fermions:
            eta = self.draw_pseudofermion(q)
            if self.prm.hasenbusch:
                eta, phi = eta
        info = hr.hr_hmc_trajectory(self.ctx, self.dims, self.prm, q, p, eta, self.work, phi=phi)
        u = torch.rand((), dtype=torch.float64, device=self.device, generator=self.gen).item()
        accept = info.dH <= 0.0 or u < math.exp(-info.dH)
        if not accept:
            q.copy_(backup)
        self.trajectories += 1
        self.accepted += int(accept)
        return accept, info
