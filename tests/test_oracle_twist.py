"""Pins of the oracle's twisted boundary conditions, psi(x + L_mu mu) = e^{i theta_mu} psi(x).

The paper (arXiv:2411.18511) does not write boundary conditions down; the
twist is the standard generalisation of the antiperiodic sign to a U(1) phase.
These tests tie the oracle's twisted operator to facts that do not come from
its boundary factor:

* free-field plane waves: momenta p_mu = (2 pi n_mu + theta_mu) / L_mu (plus
  pi / L_mu in antiperiodic directions) diagonalise D with the free symbol;
* the twist is a constant U(1) background field: with P = diag(e^{i phi(x)}),
  phi(x) = sum_mu theta_mu x_mu / L_mu, the twisted operator equals
  P D_periodic[U_mu e^{i theta_mu / L_mu}] P^+ (the periodic oracle fed U(2)
  links, a code path without any boundary factor);
* theta_mu = pi reproduces the antiperiodic bit, theta -> theta + 2 pi changes
  nothing;
* an independent dense build (tests/dense_ref.py), gamma5-hermiticity of the
  Schur operator, CG and the even-odd solve against dense solves;
* the link gradient and the force against central finite differences through
  the dense build;
* the clover operators and the clover fermion force on twisted lattices against
  dense builds and finite differences of dense-matrix actions.
"""

import numpy as np
import pytest

import oracle
import synth
from tests import dense_ref as dr

RNG = np.random.default_rng(2468)


def coords(dims):
    return np.indices(dims).reshape(4, -1).T  # [V, 4]


def rel(a, b):
    return np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))


def inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def free_field_symbol(p, m0):
    s = (m0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        s = s + 1j * np.sin(p[mu]) * dr.GAMMA[mu]
    return s


THETAS = [np.array([0.3, 0.0, 0.0, 0.0]), np.array([0.7, -1.1, 2.5, 0.4]), np.array([0.0, 0.0, 0.0, -2.9])]


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [0, 1, 12])
@pytest.mark.parametrize("k", range(len(THETAS)))
def test_free_field_twisted_plane_wave(nc, bc, k):
    theta = THETAS[k]
    dims = (4, 6, 2, 4)
    L = oracle.expand_links(dims, nc, synth.identity_links(dims))
    x = coords(dims)
    m0 = -0.1
    anti = np.array([(bc >> mu) & 1 for mu in range(4)])
    for _ in range(3):
        n = np.array([RNG.integers(0, d) for d in dims])
        p = (2 * np.pi * n + np.pi * anti + theta) / np.array(dims)
        u = RNG.normal(size=(4, nc)) + 1j * RNG.normal(size=(4, nc))
        phase = np.exp(1j * (x @ p))
        psi = phase[:, None, None] * u[None]
        want = phase[:, None, None] * (free_field_symbol(p, m0) @ u)[None]
        assert rel(oracle.dirac(dims, L, m0, psi, bc=bc, theta=theta), want) < 1e-14
        # without the twist the plane wave is no eigenvector
        assert rel(oracle.dirac(dims, L, m0, psi, bc=bc), want) > 1e-3


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [0, 9])
def test_twist_is_a_constant_u1_background(nc, bc):
    """H_theta = P H_0[U e^{i theta / L}] P^+, P = e^{i sum theta_mu x_mu / L_mu}."""
    dims = (4, 2, 4, 6)
    theta = np.array([0.9, -0.4, 1.7, 2.2])
    q = synth.haar_links(dims, 301)
    L = oracle.expand_links(dims, nc, q)
    Lb = L * np.exp(1j * theta / np.array(dims))[:, None, None, None]  # U(2) or U(1) x SO(3) links
    P = np.exp(1j * (coords(dims) @ (theta / np.array(dims))))[:, None, None]
    psi = synth.gaussian_spinor(dims, nc, 302)
    for par in (-1, 0, 1):
        got = oracle.hop(dims, L, psi, parity=par, bc=bc, theta=theta)
        want = P * oracle.hop(dims, Lb, np.conj(P) * psi, parity=par, bc=bc)
        assert rel(got, want) < 1e-14
    assert rel(oracle.hop(dims, L, psi, bc=bc), oracle.hop(dims, L, psi, bc=bc, theta=theta)) > 1e-3


def test_pi_twist_is_antiperiodic_and_2pi_is_nothing():
    dims = (4, 2, 2, 4)
    q = synth.haar_links(dims, 311)
    for nc in (2, 3):
        L = oracle.expand_links(dims, nc, q)
        psi = synth.gaussian_spinor(dims, nc, 312)
        for mu in range(4):
            th = np.zeros(4)
            th[mu] = np.pi
            assert rel(oracle.dirac(dims, L, 0.1, psi, theta=th), oracle.dirac(dims, L, 0.1, psi, bc=1 << mu)) < 1e-15
        th = np.array([0.3, -0.8, 1.1, 2.0])
        a = oracle.dirac(dims, L, 0.1, psi, bc=5, theta=th)
        b = oracle.dirac(dims, L, 0.1, psi, bc=5, theta=th + 2 * np.pi * np.array([1, -2, 0, 3]))
        assert rel(a, b) < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4), (2, 4, 2, 2)])
@pytest.mark.parametrize("bc", [0, 6])
def test_dense_bruteforce_twisted(nc, dims, bc):
    theta = np.array([0.45, 1.3, -0.7, 2.8])
    q = synth.haar_links(dims, 321)
    L = oracle.expand_links(dims, nc, q)
    D = dr.dirac_dense(dims, q, nc, 0.1, bc, theta)
    for seed in (322, 323):
        psi = synth.gaussian_spinor(dims, nc, seed)
        assert rel(oracle.dirac(dims, L, 0.1, psi, bc=bc, theta=theta).reshape(-1), D @ psi.reshape(-1)) < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_twisted_schur_complement_and_gamma5_hermiticity(nc):
    dims = (2, 4, 2, 2)
    m0, bc, theta = -0.3, 1, np.array([0.2, 0.9, -1.4, 0.6])
    q = synth.haar_links(dims, 331)
    L = oracle.expand_links(dims, nc, q)
    D = dr.dirac_dense(dims, q, nc, m0, bc, theta)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, nc, D)
    M = Dee - Deo @ np.linalg.solve(Doo, Doe)
    psi = synth.gaussian_spinor(dims, nc, 332)
    phi = synth.gaussian_spinor(dims, nc, 333)
    even = oracle.parity_mask(dims) == 0
    psi[~even] = 0
    phi[~even] = 0
    got = oracle.schur(dims, L, m0, psi, bc=bc, theta=theta).reshape(-1)
    assert rel(got[e], M @ psi.reshape(-1)[e]) < 1e-13
    assert np.all(got[o] == 0)
    gotd = oracle.schur(dims, L, m0, psi, dagger=True, bc=bc, theta=theta).reshape(-1)
    assert rel(gotd[e], M.conj().T @ psi.reshape(-1)[e]) < 1e-13
    lhs = inner(phi, oracle.schur(dims, L, m0, psi, bc=bc, theta=theta))
    rhs = inner(oracle.schur(dims, L, m0, phi, dagger=True, bc=bc, theta=theta), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    gotn = oracle.normal(dims, L, m0, psi, bc=bc, theta=theta).reshape(-1)
    assert rel(gotn[e], M.conj().T @ M @ psi.reshape(-1)[e]) < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_twisted_cg_and_eo_solve_against_dense(nc):
    dims = (4, 2, 2, 4)
    m0, bc, theta = 0.1, 1, np.array([0.35, -0.6, 1.2, 0.8])
    q = synth.haar_links(dims, 341)
    L = oracle.expand_links(dims, nc, q)
    D = dr.dirac_dense(dims, q, nc, m0, bc, theta)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, nc, D)
    M = Dee - Deo @ np.linalg.solve(Doo, Doe)
    b = synth.gaussian_spinor(dims, nc, 342)
    be = b.copy()
    be[oracle.parity_mask(dims) == 1] = 0
    x, it, tr, ok = oracle.cg(dims, L, m0, be, tol=1e-12, bc=bc, theta=theta)
    assert ok and tr <= 1e-12
    assert rel(x.reshape(-1)[e], np.linalg.solve(M.conj().T @ M, be.reshape(-1)[e])) < 1e-10
    # the even-odd solve of D x = b
    bhat = oracle.eo_source(dims, L, m0, b, bc=bc, theta=theta)
    rhs = oracle.schur(dims, L, m0, bhat, dagger=True, bc=bc, theta=theta)
    xe, it, tr, ok = oracle.cg(dims, L, m0, rhs, tol=1e-13, bc=bc, theta=theta)
    assert ok
    xf = oracle.eo_reconstruct(dims, L, m0, b, xe, bc=bc, theta=theta)
    assert rel(xf.reshape(-1), np.linalg.solve(D, b.reshape(-1))) < 1e-10


def _boundary_samples(dims, theta, n):
    """(mu, x) pairs, half of them on the boundary slice of a twisted direction."""
    V = int(np.prod(dims))
    xs = coords(dims)
    tw = [mu for mu in range(4) if theta[mu] != 0]
    out = []
    for j in range(n):
        if j % 2 == 0:
            mu = tw[RNG.integers(len(tw))]
            cands = np.where(xs[:, mu] == dims[mu] - 1)[0]
            out.append((mu, int(cands[RNG.integers(len(cands))])))
        else:
            out.append((int(RNG.integers(4)), int(RNG.integers(V))))
    return out


def _su2_exp(w):
    th = np.linalg.norm(w) / 2
    n = w / np.linalg.norm(w)
    return np.concatenate([[np.cos(th)], np.sin(th) * n])


@pytest.mark.parametrize("bc", [0, 5])
def test_twisted_link_grad_matches_finite_differences(bc):
    dims = (2, 4, 2, 4)
    theta = np.array([0.8, 0.0, -1.3, 2.1])
    q = synth.haar_links(dims, 351)
    a = synth.gaussian_spinor(dims, 2, 352)
    b = synth.gaussian_spinor(dims, 2, 353)
    G = oracle.link_grad(dims, a, b, bc=bc, theta=theta)

    def f(qq):
        return inner(a, (dr.hopping_dense(dims, qq, 2, bc, theta) @ b.reshape(-1))).real

    eps = 1e-6
    for mu, x in _boundary_samples(dims, theta, 16):
        k = RNG.integers(4)
        qp, qm = q.copy(), q.copy()
        qp[mu, x, k] += eps
        qm[mu, x, k] -= eps
        fd = (f(qp) - f(qm)) / (2 * eps)
        assert abs(fd - G[mu, x, k]) < 1e-7 * max(1.0, abs(fd)), (mu, x, k, fd, G[mu, x, k])


@pytest.mark.parametrize("bc", [0, 1])
def test_twisted_force_matches_finite_differences_of_solve_loss(bc):
    """S = Re<eta, (Mhat^+ Mhat)^-1 eta> with the twisted operator, S from dense solves."""
    dims = (2, 2, 2, 4)
    theta = np.array([1.1, -0.5, 0.0, 0.7])
    m0 = 0.2
    q = synth.haar_links(dims, 361)
    L = oracle.expand_links(dims, 2, q)
    eta = synth.gaussian_spinor(dims, 2, 362)
    even = oracle.parity_mask(dims) == 0
    eta[~even] = 0

    def S(qq):
        D = dr.dirac_dense(dims, qq, 2, m0, bc, theta)
        Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
        M = Dee - Deo @ np.linalg.solve(Doo, Doe)
        y = eta.reshape(-1)[e]
        return np.vdot(y, np.linalg.solve(M.conj().T @ M, y)).real

    kw = dict(bc=bc, theta=theta)
    X, it, tr, ok = oracle.cg(dims, L, m0, eta, tol=1e-14, maxiter=5000, **kw)
    Y = oracle.schur(dims, L, m0, X, **kw)
    Z = oracle.hop(dims, L, X, parity=1, **kw)
    W = oracle.gamma5(oracle.hop(dims, L, oracle.gamma5(Y), parity=1, **kw))
    a = np.where(even[:, None, None], Y, W)
    b = np.where(even[:, None, None], X, Z)
    F = 2.0 / (4.0 * (4 + m0)) * oracle.force(dims, L, a, b, **kw)
    eps = 1e-5
    for mu, x in _boundary_samples(dims, theta, 12):
        w = RNG.normal(size=3)
        w /= np.linalg.norm(w)
        qp, qm = q.copy(), q.copy()
        qp[mu, x] = synth.quat_mul(_su2_exp(eps * w), q[mu, x])
        qm[mu, x] = synth.quat_mul(_su2_exp(-eps * w), q[mu, x])
        fd = (S(qp) - S(qm)) / (2 * eps)
        an = F[mu, x] @ w
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (mu, x, fd, an)


def test_bad_theta_is_rejected():
    dims = (2, 2, 2, 2)
    L = oracle.expand_links(dims, 2, synth.identity_links(dims))
    psi = synth.gaussian_spinor(dims, 2, 1)
    with pytest.raises(ValueError):
        oracle.hop(dims, L, psi, theta=[0.1, np.nan, 0, 0])
    with pytest.raises(ValueError):
        oracle.hop(dims, L, psi, theta=[0.1, 0.2])


@pytest.mark.parametrize("kind", [0, 1])
def test_twisted_clover_operators_against_dense(kind):
    """The clover oracle's operators on a twisted lattice (the site term is
    blind to the twist: it sits in closed loops) against a dense build."""
    from oracle import clover as ocl

    dims = (2, 4, 2, 4)
    m0, csw, bc, theta = 0.1, 1.2, 1, np.array([0.6, -0.9, 1.4, 0.3])
    q = synth.haar_links(dims, 371)
    L = oracle.expand_links(dims, 2, q)
    A = ocl.site_term(dims, L, m0, csw, kind)
    Ad = dr.clover_site_dense(dims, q, 2, m0, csw, exponential=bool(kind))
    assert np.abs(A - Ad).max() < 1e-13
    D = dr.dirac_clover_dense(dims, q, 2, Ad, bc, theta)
    psi = synth.gaussian_spinor(dims, 2, 372)
    assert rel(ocl.dirac(dims, L, A, psi, bc=bc, theta=theta).reshape(-1), D @ psi.reshape(-1)) < 1e-14
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
    M = Dee - Deo @ np.linalg.solve(Doo, Doe)
    psi[oracle.parity_mask(dims) == 1] = 0
    got = ocl.schur(dims, L, A, psi, bc=bc, theta=theta).reshape(-1)
    assert rel(got[e], M @ psi.reshape(-1)[e]) < 1e-13


def exp_update(q, mu, x, w, eps):
    """U_mu(x) -> exp(i eps w.s/2) U_mu(x)."""
    from oracle import hmc

    out = q.copy()
    out[mu, x] = hmc.link_update(q[mu, x][None], w[None], eps)[0]
    return out


def test_twisted_clover_force_matches_finite_differences():
    """The clover fermion force (hops, site term, det A_oo) on a twisted lattice
    against finite differences of dense-matrix actions."""
    from oracle import clover as ocl

    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0, csw, bc, theta = 0.1, 1.3, 1, np.array([0.8, 0.0, -1.1, 0.5])
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, 381), dims, 0.6)
    eta = synth.gaussian_spinor(dims, 2, 382)
    odd = oracle.parity_mask(dims) == 1
    eta[odd] = 0

    def S(qq):
        A = dr.clover_site_dense(dims, qq, 2, m0, csw)
        D = dr.dirac_clover_dense(dims, qq, 2, A, bc, theta)
        Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
        M = Dee - Deo @ np.linalg.solve(Doo, Doe)
        y = eta.reshape(-1)[e]
        S_det = -2.0 * sum(np.linalg.slogdet(A[k])[1] for k in np.where(odd)[0])
        return np.vdot(y, np.linalg.solve(M.conj().T @ M, y)).real + S_det

    ferm = ocl.CloverFermions(dims, m0, csw, eta, bc=bc, tol=1e-14, theta=theta)
    S0 = S(q)
    assert abs(ferm.action(q) - S0) <= 1e-10 * abs(S0)
    F = ferm.force(q)
    eps = 1e-5
    for mu, x in _boundary_samples(dims, theta, 10):
        w = RNG.normal(size=3)
        w /= np.linalg.norm(w)
        fd = (S(exp_update(q, mu, x, w, eps)) - S(exp_update(q, mu, x, w, -eps))) / (2 * eps)
        assert abs(fd - F[mu, x] @ w) <= 1e-6 * max(1.0, abs(fd)), (mu, x, fd, F[mu, x] @ w)
