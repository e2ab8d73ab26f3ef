"""Clover and exponential-clover site terms of the Wilson-Dirac operator:
plain numpy, FP64 (test infrastructure, like the rest of ``oracle``).

The paper (arXiv:2411.18511, Sec. 2.2) names the clover improvement
(Sheikholeslami-Wohlert) and its exponential variant (Francis et al.) as an
extra site-diagonal term, precomputed per gauge field with its inverse, and
writes neither down.  The readings here are the textbook ones:

    Q_mn(x)  = the four plaquette leaves of the (mu, nu) plane that start and
               end at x, each traversed mu-first (counter-clockwise),
    F_mn(x)  = (Q_mn(x) - Q_mn(x)^+) / 8,
    s_mn     = (i/2) [g_mu, g_nu],
    C(x)     = (i/4) sum_{mu != nu} s_mn F_mn(x)     (Hermitian, 4 nc x 4 nc),
    clover:       A(x) = (4 + m0) + c_sw C(x),
    exponential:  A(x) = (4 + m0) exp(c_sw C(x) / (4 + m0)),

and the operator with the site term:

    D = A - H/2,   Mhat = A_ee - H_eo A_oo^-1 H_oe / 4,   Mhat^+ = g5 Mhat g5,
    source bhat = b_e + H_eo A_oo^-1 b_o / 2,   x_o = A_oo^-1 (b_o + H_oe x_e / 2).

Site matrices act on the (spin, colour) index s * nc + c of a spinor
[V][4][nc].  The gauge loops use the links as given (fermion boundary signs
cancel around a closed loop); the hops take the ``bc`` of the rest of the
oracle.  Library routines used as steps: ``numpy.linalg.inv`` for A_oo^-1 and
``numpy.linalg.eigh`` for the exponential of the Hermitian C.

Pinned in tests/test_oracle_clover.py: the closed form of a constant abelian
field (F_01 = i sin(B) s_3 on every site), the free field (A = 4 + m0),
Hermiticity and chirality of A, gauge covariance, and an independent dense
build (tests/dense_ref.py).  The HMC force of the clover term (bottom of this
file: the derivative through the leaves, the pseudofermion and det A_oo
terms) is pinned in tests/test_oracle_clover_force.py by finite differences,
the whole force against dense-matrix actions.
"""

from __future__ import annotations

import numpy as np

KIND_SW, KIND_EXP = 0, 1


def _gammas():
    from . import gamma  # the oracle's own table

    return [gamma(mu) for mu in range(4)]


def sigma(mu: int, nu: int) -> np.ndarray:
    """s_mn = (i/2) [g_mu, g_nu] (4 x 4, Hermitian)."""
    g = _gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def _neighbours(dims):
    """fwd[mu][x] = x + mu-hat and bwd[mu][x] = x - mu-hat (periodic)."""
    idx = np.arange(int(np.prod(dims))).reshape(dims)
    fwd = [np.roll(idx, -1, axis=mu).reshape(-1) for mu in range(4)]
    bwd = [np.roll(idx, 1, axis=mu).reshape(-1) for mu in range(4)]
    return fwd, bwd


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum("xab,xbc->xac", out, m)
    return out


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def clover_leaves(dims, L, mu: int, nu: int) -> np.ndarray:
    """Q_mn(x) for every site: [V, nc, nc]."""
    fwd, bwd = _neighbours(dims)
    Um, Un = L[mu], L[nu]
    f, b = fwd, bwd
    xpm, xpn = f[mu], f[nu]
    xmm, xmn = b[mu], b[nu]
    xmm_pn = f[nu][xmm]       # x - mu + nu
    xmm_mn = b[nu][xmm]       # x - mu - nu
    xmn_pm = f[mu][xmn]       # x - nu + mu
    q = _mm(Um, Un[xpm], _dag(Um[xpn]), _dag(Un))
    q = q + _mm(Un, _dag(Um[xmm_pn]), _dag(Un[xmm]), Um[xmm])
    q = q + _mm(_dag(Um[xmm]), _dag(Un[xmm_mn]), Um[xmm_mn], Un[xmn])
    q = q + _mm(_dag(Un[xmn]), Um[xmn], Un[xmn_pm], _dag(Um))
    return q


def field_strength(dims, L) -> np.ndarray:
    """F[mu, nu] = (Q_mn - Q_mn^+) / 8, shape [4, 4, V, nc, nc] (zero for mu = nu)."""
    V, nc = L.shape[1], L.shape[-1]
    F = np.zeros((4, 4, V, nc, nc), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                Q = clover_leaves(dims, L, mu, nu)
                F[mu, nu] = (Q - _dag(Q)) / 8.0
    return F


def clover_generator(dims, L) -> np.ndarray:
    """C(x) = (i/4) sum_{mu != nu} s_mn (x) F_mn(x), shape [V, 4 nc, 4 nc]."""
    F = field_strength(dims, L)
    V, nc = L.shape[1], L.shape[-1]
    C = np.zeros((V, 4, nc, 4, nc), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                C += 0.25j * np.einsum("st,xab->xsatb", sigma(mu, nu), F[mu, nu])
    return C.reshape(V, 4 * nc, 4 * nc)


def site_term(dims, L, m0: float, csw: float, kind: int = KIND_SW) -> np.ndarray:
    """A(x) for every site, [V, 4 nc, 4 nc]."""
    C = clover_generator(dims, L)
    n = C.shape[-1]
    a = 4.0 + m0
    if kind == KIND_SW:
        return a * np.eye(n)[None] + csw * C
    if kind != KIND_EXP:
        raise ValueError("kind: KIND_SW or KIND_EXP")
    # exp of the Hermitian csw C / a from its eigen-decomposition
    w, U = np.linalg.eigh(csw * C / a)
    return a * np.einsum("xij,xj,xkj->xik", U, np.exp(w), np.conj(U))


def apply_site(A, psi) -> np.ndarray:
    """(A psi)(x) = A(x) psi(x) for a spinor [V, 4, nc]."""
    V, _, nc = psi.shape
    return np.einsum("xij,xj->xi", A, psi.reshape(V, 4 * nc)).reshape(V, 4, nc)


def _parity(dims):
    from . import parity_mask

    return parity_mask(dims)


def dirac(dims, L, A, psi, bc=None, theta=None) -> np.ndarray:
    """D psi = A psi - H psi / 2 on all sites."""
    from . import hop

    psi = np.asarray(psi, dtype=np.complex128)
    return apply_site(A, psi) - 0.5 * hop(dims, L, psi, bc=bc, theta=theta)


def schur(dims, L, A, psi, dagger: bool = False, bc=None, theta=None) -> np.ndarray:
    """Mhat psi (or Mhat^+ psi) on the even sites of a full-lattice array; odd sites -> 0."""
    from . import gamma5, hop

    par = _parity(dims)
    even, odd = par == 0, par == 1
    inp = np.array(psi, dtype=np.complex128)
    inp[odd] = 0
    if dagger:
        inp = gamma5(inp)
    t = hop(dims, L, inp, parity=1, bc=bc, theta=theta)           # H_oe in (odd sites)
    Ainv = np.linalg.inv(A[odd])
    t[odd] = apply_site(Ainv, t[odd])                 # A_oo^-1 H_oe in
    u = hop(dims, L, t, parity=0, bc=bc, theta=theta)              # H_eo A_oo^-1 H_oe in
    out = np.zeros_like(inp)
    out[even] = apply_site(A[even], inp[even]) - 0.25 * u[even]
    if dagger:
        out = gamma5(out)
    return out


def normal(dims, L, A, psi, bc=None, theta=None) -> np.ndarray:
    """Mhat^+ Mhat psi on even sites."""
    return schur(dims, L, A, schur(dims, L, A, psi, bc=bc, theta=theta), dagger=True, bc=bc, theta=theta)


def cg(dims, L, A, b, tol: float = 1e-10, maxiter: int = 10000, bc=None, theta=None):
    """Hestenes-Stiefel CG on Mhat^+ Mhat x = b (even sites) from x = 0.
    Returns (x, iters, true_rel_residual, converged)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    p = b.copy()
    bb = np.vdot(b, b).real
    rr = bb
    it = 0
    while it < maxiter and np.sqrt(rr / bb) > tol:
        q = normal(dims, L, A, p, bc=bc, theta=theta)
        alpha = rr / np.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    true = np.linalg.norm(b - normal(dims, L, A, x, bc=bc, theta=theta)) / np.sqrt(bb)
    return x, it, true, bool(np.sqrt(rr / bb) <= tol)


def eo_source(dims, L, A, b, bc=None, theta=None) -> np.ndarray:
    """bhat_e = b_e - D_eo A_oo^-1 b_o = b_e + H_eo A_oo^-1 b_o / 2; odd sites zero."""
    from . import hop

    par = _parity(dims)
    odd = par == 1
    t = np.zeros_like(np.asarray(b, dtype=np.complex128))
    t[odd] = apply_site(np.linalg.inv(A[odd]), np.asarray(b, dtype=np.complex128)[odd])
    out = np.array(b, dtype=np.complex128) + 0.5 * hop(dims, L, t, parity=0, bc=bc, theta=theta)
    out[odd] = 0
    return out


def eo_reconstruct(dims, L, A, b, xe, bc=None, theta=None) -> np.ndarray:
    """x_o = A_oo^-1 (b_o - D_oe x_e) = A_oo^-1 (b_o + H_oe x_e / 2); returns the full x."""
    from . import hop

    odd = _parity(dims) == 1
    h = hop(dims, L, np.asarray(xe, dtype=np.complex128), parity=1, bc=bc, theta=theta)
    x = np.array(xe, dtype=np.complex128)
    x[odd] = apply_site(np.linalg.inv(A[odd]), np.asarray(b, dtype=np.complex128)[odd] + 0.5 * h[odd])
    return x


# ---------------------------------------------------------------- link derivatives (fundamental)
#
# The HMC force of the clover term (SW form).  With the site term in the
# even-odd operator, Mhat = A_ee - H_eo A_oo^-1 H_oe / 4, two flavours weigh
# det(D^+ D) = det(A_oo)^2 det(Mhat^+ Mhat): the pseudofermion action
# S_pf = Re <eta, (Mhat^+ Mhat)^-1 eta> and S_det = -2 sum_{x odd} log det A(x).
# With X = (Mhat^+ Mhat)^-1 eta, Y = Mhat X, Z = A_oo^-1 H_oe X and
# W = A_oo^-1 H_eo^+ Y (odd sites), dS_pf = -2 Re <Y, dMhat X> splits into
#   the hops:       1/2 d Re <a, H b>,  a = (Y, W), b = (X, Z),
#   the site term:  Re sum_x tr[dA(x) Lam(x)],  Lam = -2 X Y^+ (even), -1/2 Z W^+ (odd),
# and dS_det = Re sum_x tr[dA(x) Lam_det(x)], Lam_det = -2 A(x)^-1 (odd).
# dA = c_sw dC, and C depends on the links through the leaves of F_mn.

_T = [0.5j * np.array([[0, 1], [1, 0]], dtype=complex), 0.5j * np.array([[0, -1j], [1j, 0]]),
      0.5j * np.array([[1, 0], [0, -1]], dtype=complex)]  # generators i s_a / 2


def _leaf_factors(mu: int, nu: int):
    """The four leaves of Q_mn(x), as in ``clover_leaves``: lists of
    (direction, (steps along mu, steps along nu) from x, daggered)."""
    return [[(mu, (0, 0), False), (nu, (1, 0), False), (mu, (0, 1), True), (nu, (0, 0), True)],
            [(nu, (0, 0), False), (mu, (-1, 1), True), (nu, (-1, 0), True), (mu, (-1, 0), False)],
            [(mu, (-1, 0), True), (nu, (-1, -1), True), (mu, (-1, -1), False), (nu, (0, -1), False)],
            [(nu, (0, -1), True), (mu, (0, -1), False), (nu, (1, -1), False), (mu, (0, 0), True)]]


def clover_derivative(dims, L, Lam) -> np.ndarray:
    """G[rho, z, a] = d/dw_a Re sum_y tr[C(y) Lam(y)] under U_rho(z) -> exp(i w.s/2) U_rho(z),
    fundamental links L [4, V, 2, 2], Lam [V, 8, 8] (index s * 2 + c).

    tr[C Lam] = (i/2) sum_{mu<nu} tr_c[F_mn K_mn] with K_mn = tr_s[(s_mn (x) 1) Lam]
    (the mu > nu terms repeat the mu < nu ones), F_mn = (Q_mn - Q_mn^+) / 8.  For a
    leaf P = A V B whose factor V is the varied link U (V = U) or its inverse
    (V = U^+), dU = X U with X = i w.s/2 anti-Hermitian, and
      tr[dP K] - tr[dP^+ K] = tr[X (U B K A + A^+ K B^+ U^+)]      (V = U),
                            = -tr[X (B K A U^+ + U A^+ K B^+)]     (V = U^+),
    so each occurrence adds Re[(i/16) tr(T_a G)] to the link's component a."""
    V = L.shape[1]
    fwd, bwd = _neighbours(dims)
    Lam = np.asarray(Lam, dtype=np.complex128).reshape(V, 4, 2, 4, 2)
    G = np.zeros((4, V, 3))
    eye = np.broadcast_to(np.eye(2, dtype=complex), (V, 2, 2))

    def site(mu, nu, a, b):
        """index of y + a mu-hat + b nu-hat for every y"""
        idx = np.arange(V)
        for _ in range(abs(a)):
            idx = (fwd if a > 0 else bwd)[mu][idx]
        for _ in range(abs(b)):
            idx = (fwd if b > 0 else bwd)[nu][idx]
        return idx

    for mu in range(4):
        for nu in range(mu + 1, 4):
            K = np.einsum("st,xtbsa->xba", sigma(mu, nu), Lam)   # K_mn(y)[b, a]
            for leaf in _leaf_factors(mu, nu):
                where = [site(mu, nu, a, b) for _, (a, b), _ in leaf]
                mats = [(_dag(L[d][z]) if dag else L[d][z]) for (d, _, dag), z in zip(leaf, where)]
                for k, (d, _, dag) in enumerate(leaf):
                    A = _mm(eye, *mats[:k])
                    B = _mm(eye, *mats[k + 1:])
                    U = L[d][where[k]]
                    if not dag:
                        Gm = _mm(U, B, K, A) + _mm(_dag(A), K, _dag(B), _dag(U))
                    else:
                        Gm = -(_mm(B, K, A, _dag(U)) + _mm(U, _dag(A), K, _dag(B)))
                    for a in range(3):
                        val = np.real(1j / 16.0 * np.einsum("ij,xji->x", _T[a], Gm))
                        np.add.at(G[d, :, a], where[k], val)
    return G


def exp_insertion(A, Lam, m0: float) -> np.ndarray:
    """The insertion that carries an exponential site term's variation to C:
    for A = a exp(X), a = 4 + m0, X = c_sw C / a,
      d Re tr[A Lam] = c_sw Re tr[dC Lam'],  Lam' = int_0^1 exp((1-s) X) Lam exp(s X) ds
    (dA = a int_0^1 exp(s X) dX exp((1-s) X) ds and the trace is cyclic).  In the
    eigenbasis of X (that of A, eigenvalues mu = a e^lambda) the integral is the
    divided difference of exp: (V^+ Lam' V)_ij = (V^+ Lam V)_ij (e^l_i - e^l_j) / (l_i - l_j),
    i.e. the logarithmic mean of mu_i and mu_j over a.  Per chiral block (C and A
    are block diagonal, so only the diagonal blocks of Lam' enter); Lam [V, 8, 8]."""
    A = np.asarray(A)
    Lam = np.asarray(Lam, dtype=np.complex128)
    out = np.zeros_like(Lam)
    a = 4.0 + m0
    n = A.shape[-1] // 2
    for b in range(2):
        sl = slice(b * n, (b + 1) * n)
        mu, V = np.linalg.eigh(A[:, sl, sl])
        lam = np.log(mu / a)
        li, lj = lam[:, :, None], lam[:, None, :]
        d = li - lj
        with np.errstate(invalid="ignore", divide="ignore"):
            phi = np.where(np.abs(d) > 1e-8, (np.exp(li) - np.exp(lj)) / d, np.exp(0.5 * (li + lj)))
        Lt = np.einsum("xki,xkl,xlj->xij", np.conj(V), Lam[:, sl, sl], V)
        out[:, sl, sl] = np.einsum("xik,xkl,xjl->xij", V, Lt * phi, np.conj(V))
    return out


def det_action(A, dims) -> float:
    """S_det = -2 sum_{x odd} log det A(x) (A Hermitian positive definite)."""
    from . import parity_mask

    odd = parity_mask(dims) == 1
    sign, logdet = np.linalg.slogdet(A[odd])
    assert np.all(sign.real > 0)
    return float(-2.0 * np.sum(logdet.real))


class CloverFermions:
    """Two flavours of clover fermions through the even-odd pseudofermion:
    S = S_pf + S_det (see above) and its su(2) force, for HMC trajectories
    (``oracle.hmc.trajectory`` takes it as its ``fermions``).  kind KIND_SW or
    KIND_EXP; for the exponential form log det A = N log(4 + m0) + tr X is a
    constant (C is traceless), so S_det has no force, and the site term's force
    takes the insertion through ``exp_insertion``."""

    def __init__(self, dims, m0: float, csw: float, eta, bc=0, tol: float = 1e-13, theta=None, kind=KIND_SW):
        self.dims, self.m0, self.csw, self.eta, self.bc, self.tol, self.theta = dims, m0, csw, eta, bc, tol, theta
        self.kind = kind
        self.iters = 0

    def _setup(self, q):
        from . import expand_links

        L = expand_links(self.dims, 2, q)
        A = site_term(self.dims, L, self.m0, self.csw, self.kind)
        return L, A

    def solve(self, q):
        L, A = self._setup(q)
        x, it, tr, ok = cg(self.dims, L, A, self.eta, tol=self.tol, maxiter=50000, bc=self.bc, theta=self.theta)
        assert ok, tr
        self.iters += it
        return L, A, x

    def action(self, q) -> float:
        L, A, x = self.solve(q)
        return float(np.vdot(self.eta, x).real) + det_action(A, self.dims)

    def force(self, q) -> np.ndarray:
        L, A, X = self.solve(q)
        return self.force_at(q, X)

    def force_at(self, q, X, det: bool = True, Y=None) -> np.ndarray:
        """The force for a given even X (X = (Mhat^+ Mhat)^-1 eta in the HMC;
        det=False leaves out the det A_oo term): the derivative of
        -2 Re <Y, dMhat X> with Y = Mhat X, or the given even Y."""
        from . import force, gamma5, hop, parity_mask

        L, A = self._setup(q)
        X = np.asarray(X, dtype=np.complex128)
        d, kw = self.dims, dict(bc=self.bc, theta=self.theta)
        odd = parity_mask(d) == 1
        Ainv = np.zeros_like(A)
        Ainv[odd] = np.linalg.inv(A[odd])
        Y = schur(d, L, A, X, **kw) if Y is None else np.asarray(Y, dtype=np.complex128)
        Z = apply_site(Ainv, hop(d, L, X, parity=1, **kw))                       # A_oo^-1 H_oe X
        W = apply_site(Ainv, gamma5(hop(d, L, gamma5(Y), parity=1, **kw)))     # A_oo^-1 H_eo^+ Y
        a = np.where(odd[:, None, None], W, Y)
        b = np.where(odd[:, None, None], Z, X)
        F = 0.5 * force(d, L, a, b, **kw)
        V = X.shape[0]
        outer = lambda u, v: np.einsum("xi,xj->xij", u.reshape(V, 8), np.conj(v.reshape(V, 8)))  # noqa: E731
        if self.kind == KIND_EXP:
            Lam = np.where(odd[:, None, None], -0.5 * outer(Z, W), -2.0 * outer(X, Y))
            return F + self.csw * clover_derivative(d, L, exp_insertion(A, Lam, self.m0))
        Lam = np.where(odd[:, None, None], -0.5 * outer(Z, W) - (2.0 * Ainv if det else 0.0), -2.0 * outer(X, Y))
        return F + self.csw * clover_derivative(d, L, Lam)


class CloverHasenbusch:
    """Clover fermions with Hasenbusch's mass preconditioning: with Mhat_H the
    clover Schur operator at the heavier mass m0_h (same C, A_H = (4 + m0_h) +
    c_sw C, or its exponential),
      S = Re <eta, (Mhat_H^+ Mhat_H)^-1 eta> + Re <eta2, (Mhat^+ Mhat)^-1 eta2>
          - 2 sum_{x odd} log det A(x),     eta2 = Mhat_H^+ phi,
    the det term at the light mass (det D = det A_oo det Mhat, and det Mhat^+ Mhat
    = det Mhat_H^+ Mhat_H times the ratio).  The variation of eta2 adds
    2 Re <phi, dMhat_H X2>, i.e. minus the force of -2 Re <Y, dMhat_H X> at
    X = X2, Y = phi."""

    def __init__(self, dims, m0: float, m0_h: float, csw: float, eta, phi, bc=0, tol: float = 1e-13, theta=None,
                 kind=KIND_SW):
        self.dims, self.m0, self.m0_h, self.csw, self.bc, self.tol, self.theta = dims, m0, m0_h, csw, bc, tol, theta
        self.heavy = CloverFermions(dims, m0_h, csw, eta, bc=bc, tol=tol, theta=theta, kind=kind)
        self.light = CloverFermions(dims, m0, csw, None, bc=bc, tol=tol, theta=theta, kind=kind)
        self.phi = np.asarray(phi, dtype=np.complex128)
        self.iters = 0

    def _ratio(self, q):
        Lh, Ah = self.heavy._setup(q)
        kw = dict(bc=self.bc, theta=self.theta)
        eta2 = schur(self.dims, Lh, Ah, self.phi, dagger=True, **kw)
        L, A = self.light._setup(q)
        x, it, tr, ok = cg(self.dims, L, A, eta2, tol=self.tol, maxiter=50000, **kw)
        assert ok, tr
        self.iters += it
        return A, eta2, x

    def action(self, q) -> float:
        _, _, Xh = self.heavy.solve(q)
        A, eta2, X2 = self._ratio(q)
        return (float(np.vdot(self.heavy.eta, Xh).real) + float(np.vdot(eta2, X2).real)
                + det_action(A, self.dims))

    def force(self, q) -> np.ndarray:
        _, _, Xh = self.heavy.solve(q)
        _, _, X2 = self._ratio(q)
        return (self.heavy.force_at(q, Xh, det=False) + self.light.force_at(q, X2, det=True)
                - self.heavy.force_at(q, X2, det=False, Y=self.phi))
