"""Hybrid Monte Carlo molecular dynamics for SU(2) with two flavours of
even-odd preconditioned Wilson fermions: plain numpy, FP64 (test
infrastructure, like the rest of ``oracle``).

The paper (arXiv:2411.18511, Sec. 1 and Sec. 2.1) names HMC as the consumer of
the even-odd operator and of its inverters, and prints none of its formulas.
The readings here are the textbook ones:

* Gauge action (Wilson plaquette, SU(2)):
  ``S_g = beta sum_{x, mu<nu} (1 - 1/2 Re tr P_mn(x))``.
* Pseudofermion action on even sites: ``S_f = Re <eta, (Mhat^+ Mhat)^-1 eta>``,
  drawn as ``eta = Mhat^+ xi`` with ``P(xi) ~ exp(-xi^+ xi)``.
* Momenta p_a(x, mu), a = 1..3, kinetic energy ``1/2 sum p_a^2``; the flow
  ``dU/dt = i (p.s/2) U``, ``dp_a/dt = -F_a`` with ``F_a = dS/dw_a`` under
  ``U -> exp(i w.s/2) U`` conserves ``H = 1/2 sum p^2 + S_g + S_f``.
* Integrators: leapfrog (half momentum steps at the ends) and Omelyan's
  second-order minimum-norm scheme (lambda = 0.1931833275037836).
* Hasenbusch mass preconditioning: two pseudofermions, one at a heavier mass
  and one for the ratio of the two determinants (class ``Hasenbusch``).
* Multiple time scales (Sexton and Weingarten): with ``n_steps_gauge = m > 1``
  the pseudofermion force moves the momenta on the outer integrator and every
  outer link update of length t becomes m steps of the same integrator, of
  length t/m, driven by the gauge force alone.

Pinned in tests/test_oracle_hmc.py: the gauge force against central finite
differences of S_g, the link update against a matrix exponential,
reversibility of both integrators, second-order scaling of Delta H with the
step size, and the fermion part through ``oracle.force`` (pinned by finite
differences of a dense solve in tests/test_oracle_pins.py); the two-level
scheme against the single-level integrator (a vanishing outer force, and one
inner leapfrog step), its reversibility and its second order.
"""

from __future__ import annotations

import numpy as np

LEAPFROG, OMELYAN = 0, 1
OMELYAN_LAMBDA = 0.1931833275037836

_SIG = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
        np.array([[1, 0], [0, -1]], dtype=complex)]


def _su2(q):
    """2x2 matrices a0 + i a.s of quaternions [..., 4]."""
    a0, a1, a2, a3 = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    m = np.empty(q.shape[:-1] + (2, 2), dtype=complex)
    m[..., 0, 0] = a0 + 1j * a3
    m[..., 0, 1] = a2 + 1j * a1
    m[..., 1, 0] = -a2 + 1j * a1
    m[..., 1, 1] = a0 - 1j * a3
    return m


def _quat(m):
    """Quaternion of a 2x2 matrix of the form a0 + i a.s."""
    return np.stack([m[..., 0, 0].real, m[..., 0, 1].imag, m[..., 0, 1].real, m[..., 0, 0].imag], axis=-1)


def _shift(dims, mu, step):
    idx = np.arange(int(np.prod(dims))).reshape(dims)
    return np.roll(idx, -step, axis=mu).reshape(-1)


def gauge_action(dims, q, beta: float) -> float:
    """S_g = beta sum_{x, mu<nu} (1 - 1/2 Re tr P_mn(x)), from the oracle's plaquette."""
    from . import plaquette

    V = int(np.prod(dims))
    return beta * 6 * V * (1.0 - plaquette(dims, q))


def staples(dims, q, mu: int) -> np.ndarray:
    """V_mu(x) = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)],
    so that every plaquette containing U_mu(x) is tr(U_mu(x) V_mu(x)) (summed): [V, 2, 2]."""
    U = _su2(q)
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))  # noqa: E731
    mm = lambda a, b: np.einsum("xab,xbc->xac", a, b)  # noqa: E731
    fm = _shift(dims, mu, 1)
    S = np.zeros((U.shape[1], 2, 2), dtype=complex)
    for nu in range(4):
        if nu == mu:
            continue
        fn, bn = _shift(dims, nu, 1), _shift(dims, nu, -1)
        fm_bn = _shift(dims, nu, -1)[fm]  # x + mu - nu
        S += mm(mm(U[nu][fm], dag(U[mu][fn])), dag(U[nu]))
        S += mm(mm(dag(U[nu][fm_bn]), dag(U[mu][bn])), U[nu][bn])
    return S


def gauge_force(dims, q, beta: float) -> np.ndarray:
    """F[mu, x, a] = dS_g/dw_a under U_mu(x) -> exp(i w.s/2) U_mu(x):
    S_g holds U_mu(x) as -beta/2 Re tr(U V) + const, so F_a = -beta/2 Re tr((i s_a/2) U V)."""
    U = _su2(q)
    F = np.zeros((4, U.shape[1], 3))
    for mu in range(4):
        W = np.einsum("xab,xbc->xac", U[mu], staples(dims, q, mu))
        for a in range(3):
            F[mu, :, a] = -0.5 * beta * np.einsum("ab,xba->x", 0.5j * _SIG[a], W).real
    return F


def link_update(q, p, eps: float) -> np.ndarray:
    """U -> exp(i eps p.s/2) U for every link (exp(i t n.s) = cos t + i sin t n.s)."""
    norm = np.linalg.norm(p, axis=-1)
    th = 0.5 * eps * norm
    with np.errstate(invalid="ignore", divide="ignore"):
        n = np.where(norm[..., None] > 0, p / norm[..., None], 0.0)
    E = np.zeros(q.shape[:-1] + (2, 2), dtype=complex)
    E[..., 0, 0] = np.cos(th)
    E[..., 1, 1] = np.cos(th)
    for a in range(3):
        E += 1j * (np.sin(th) * n[..., a])[..., None, None] * _SIG[a]
    return _quat(np.einsum("...ab,...bc->...ac", E, _su2(q)))


def kinetic(p) -> float:
    return 0.5 * float(np.sum(p * p))


class Fermions:
    """The pseudofermion part for the links q: S_f and its force (one CG solve)."""

    def __init__(self, dims, m0: float, eta, bc=0, tol: float = 1e-13, theta=None):
        self.dims, self.m0, self.eta, self.bc, self.tol, self.theta = dims, m0, eta, bc, tol, theta
        self.iters = 0

    def solve(self, q):
        from . import cg, expand_links

        L = expand_links(self.dims, 2, q)
        x, it, tr, ok = cg(self.dims, L, self.m0, self.eta, tol=self.tol, maxiter=50000, bc=self.bc, theta=self.theta)
        assert ok, tr
        self.iters += it
        return L, x

    def action(self, q) -> float:
        _, x = self.solve(q)
        return float(np.vdot(self.eta, x).real)

    def force(self, q) -> np.ndarray:
        """dS_f/dw = 2c dRe<a, H b>/dw with a = (Y, H_eo^+ Y), b = (X, H_oe X), X = (Mhat^+ Mhat)^-1 eta,
        Y = Mhat X, c = 1/(4 (4+m0))."""
        from . import force, gamma5, hop, parity_mask, schur

        L, X = self.solve(q)
        d, bc = self.dims, self.bc
        Y = schur(d, L, self.m0, X, bc=bc, theta=self.theta)
        Z = hop(d, L, X, parity=1, bc=bc, theta=self.theta)
        W = gamma5(hop(d, L, gamma5(Y), parity=1, bc=bc, theta=self.theta))
        even = parity_mask(d) == 0
        a = np.where(even[:, None, None], Y, W)
        b = np.where(even[:, None, None], X, Z)
        return 2.0 / (4.0 * (4.0 + self.m0)) * force(d, L, a, b, bc=bc, theta=self.theta)


class Hasenbusch:
    """Two flavours through Hasenbusch's mass preconditioning (two pseudofermions):
    det(Mhat^+ Mhat) = det(Mhat_H^+ Mhat_H) det[(Mhat^+ Mhat) / (Mhat_H^+ Mhat_H)],
    S = Re <eta, (Mhat_H^+ Mhat_H)^-1 eta> + Re <eta2, (Mhat^+ Mhat)^-1 eta2>,
    eta2 = Mhat_H^+ phi (it depends on the links), Mhat_H the Schur operator at
    the heavier mass m0_h.  The heat bath draws eta = Mhat_H^+ xi1 and
    phi = Mhat_H (Mhat_H^+ Mhat_H)^-1 Mhat^+ xi2, so that S = |xi1|^2 + |xi2|^2.
    The force of the second term adds, to the usual one, the variation of eta2:
    2 Re <X2, dMhat_H^+ phi> = -2 c_H dRe <a', H b'> with a' = (g5 X2, H_eo^+ g5 X2),
    b' = (g5 phi, H_oe g5 phi), c_H = 1/(4 (4 + m0_h))."""

    def __init__(self, dims, m0: float, m0_h: float, eta, phi, bc=0, tol: float = 1e-13, theta=None):
        self.dims, self.m0, self.m0_h, self.bc, self.tol, self.theta = dims, m0, m0_h, bc, tol, theta
        self.heavy = Fermions(dims, m0_h, eta, bc=bc, tol=tol, theta=theta)
        self.phi = np.asarray(phi, dtype=np.complex128)
        self.iters = 0

    def _eta2(self, L):
        from . import schur

        return schur(self.dims, L, self.m0_h, self.phi, dagger=True, bc=self.bc, theta=self.theta)

    def _ratio(self, q):
        from . import cg, expand_links

        L = expand_links(self.dims, 2, q)
        eta2 = self._eta2(L)
        x, it, tr, ok = cg(self.dims, L, self.m0, eta2, tol=self.tol, maxiter=50000, bc=self.bc, theta=self.theta)
        assert ok, tr
        self.iters += it
        return L, eta2, x

    def action(self, q) -> float:
        _, eta2, x = self._ratio(q)
        return self.heavy.action(q) + float(np.vdot(eta2, x).real)

    def force(self, q) -> np.ndarray:
        from . import force, gamma5, hop, parity_mask, schur

        L, eta2, X = self._ratio(q)
        d, bc = self.dims, self.bc
        even = parity_mask(d) == 0

        def pair(u, v):
            """a = (u, H_eo^+ u), b = (v, H_oe v) as full fields."""
            W = gamma5(hop(d, L, gamma5(u), parity=1, bc=bc, theta=self.theta))
            Z = hop(d, L, v, parity=1, bc=bc, theta=self.theta)
            return np.where(even[:, None, None], u, W), np.where(even[:, None, None], v, Z)

        a, b = pair(schur(d, L, self.m0, X, bc=bc, theta=self.theta), X)
        F = 2.0 / (4.0 * (4.0 + self.m0)) * force(d, L, a, b, bc=bc, theta=self.theta)
        a2, b2 = pair(gamma5(X), gamma5(self.phi))
        F = F - 2.0 / (4.0 * (4.0 + self.m0_h)) * force(d, L, a2, b2, bc=bc, theta=self.theta)
        return F + self.heavy.force(q)


def trajectory(dims, q, p, beta: float, n_steps: int, tau: float, integrator: int = LEAPFROG, fermions=None,
               n_steps_gauge: int = 1):
    """One MD trajectory from (q, p).  Returns (q, p, info) with info holding
    H at both ends and its parts.  n_steps_gauge > 1 (with fermions): two time
    scales, see ``nested_steps``."""
    q = np.array(q, dtype=float)
    p = np.array(p, dtype=float)
    eps = tau / n_steps
    if fermions is not None and n_steps_gauge > 1:
        H0, parts0 = _hamiltonian(dims, q, p, beta, fermions)
        q, p = nested_steps(dims, q, p, beta, n_steps, eps, integrator, fermions, n_steps_gauge)
        H1, parts1 = _hamiltonian(dims, q, p, beta, fermions)
        return q, p, {"H0": H0, "H1": H1, "dH": H1 - H0, "start": parts0, "end": parts1}

    def force(qq):
        F = gauge_force(dims, qq, beta)
        if fermions is not None:
            F = F + fermions.force(qq)
        return F

    def hamiltonian(qq, pp):
        parts = {"kinetic": kinetic(pp), "gauge": gauge_action(dims, qq, beta),
                 "fermion": fermions.action(qq) if fermions is not None else 0.0}
        return sum(parts.values()), parts

    H0, parts0 = hamiltonian(q, p)
    if integrator == LEAPFROG:
        for _ in range(n_steps):
            p = p - 0.5 * eps * force(q)
            q = link_update(q, p, eps)
            p = p - 0.5 * eps * force(q)
    elif integrator == OMELYAN:
        lam = OMELYAN_LAMBDA
        for _ in range(n_steps):
            p = p - lam * eps * force(q)
            q = link_update(q, p, 0.5 * eps)
            p = p - (1.0 - 2.0 * lam) * eps * force(q)
            q = link_update(q, p, 0.5 * eps)
            p = p - lam * eps * force(q)
    else:
        raise ValueError("integrator: LEAPFROG or OMELYAN")
    H1, parts1 = hamiltonian(q, p)
    return q, p, {"H0": H0, "H1": H1, "dH": H1 - H0, "start": parts0, "end": parts1}


def _hamiltonian(dims, q, p, beta, fermions):
    parts = {"kinetic": kinetic(p), "gauge": gauge_action(dims, q, beta), "fermion": fermions.action(q)}
    return sum(parts.values()), parts


def _gauge_steps(dims, q, p, beta, t, m, integrator):
    """The inner level: m steps of length t/m driven by the gauge force alone."""
    h = t / m
    lam = OMELYAN_LAMBDA
    for _ in range(m):
        if integrator == LEAPFROG:
            p = p - 0.5 * h * gauge_force(dims, q, beta)
            q = link_update(q, p, h)
            p = p - 0.5 * h * gauge_force(dims, q, beta)
        else:
            p = p - lam * h * gauge_force(dims, q, beta)
            q = link_update(q, p, 0.5 * h)
            p = p - (1.0 - 2.0 * lam) * h * gauge_force(dims, q, beta)
            q = link_update(q, p, 0.5 * h)
            p = p - lam * h * gauge_force(dims, q, beta)
    return q, p


def nested_steps(dims, q, p, beta, n_steps, eps, integrator, fermions, m):
    """The outer level: n_steps steps of length eps whose momentum kicks use the
    pseudofermion force alone and whose link updates of length t are m inner
    steps of length t/m (``_gauge_steps``), same integrator on both levels."""
    if integrator not in (LEAPFROG, OMELYAN):
        raise ValueError("integrator: LEAPFROG or OMELYAN")
    lam = OMELYAN_LAMBDA
    for _ in range(n_steps):
        if integrator == LEAPFROG:
            p = p - 0.5 * eps * fermions.force(q)
            q, p = _gauge_steps(dims, q, p, beta, eps, m, integrator)
            p = p - 0.5 * eps * fermions.force(q)
        else:
            p = p - lam * eps * fermions.force(q)
            q, p = _gauge_steps(dims, q, p, beta, 0.5 * eps, m, integrator)
            p = p - (1.0 - 2.0 * lam) * eps * fermions.force(q)
            q, p = _gauge_steps(dims, q, p, beta, 0.5 * eps, m, integrator)
            p = p - lam * eps * fermions.force(q)
    return q, p
