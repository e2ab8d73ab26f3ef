"""Pins of the CPU oracle against facts that do not come from the oracle itself.

The paper (arXiv:2411.18511) names the unimproved Wilson-Dirac operator and its
even-odd preconditioned form (Sec. 2.1, Table 1) without printing a formula or
a worked example, so the oracle is pinned by closed forms and invariants of
that operator:

* free-field plane waves: D e^{ipx} u = [m0 + sum(1-cos p) + i sum g sin p] e^{ipx} u,
  with p_mu = 2 pi n / L_mu, or (2n+1) pi / L_mu in antiperiodic directions
* flat non-trivial connections (momentum shifted by the link's eigenphases)
* gamma5-hermiticity, gauge covariance
* brute force against an independent dense build (tests/dense_ref.py), on
  lattices with extent-2 directions where forward and backward hops coincide
* Schur-complement identities of the even-odd split
* CG against a dense solve
* link derivatives against central finite differences
"""

import numpy as np
import pytest

import oracle
import synth
from tests import dense_ref as dr

RNG = np.random.default_rng(12345)


def coords(dims):
    return np.indices(dims).reshape(4, -1).T  # [V, 4]


def inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def rel(a, b):
    return np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))


# ---------------------------------------------------------------- gamma algebra

def test_gamma_basis_is_chiral_and_clifford():
    g = [oracle.gamma(mu) for mu in range(4)]
    for mu in range(4):
        np.testing.assert_array_equal(g[mu], dr.GAMMA[mu])
        np.testing.assert_allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            np.testing.assert_allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    g5 = oracle.gamma(4)
    np.testing.assert_allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    np.testing.assert_allclose(g5, np.diag([-1, -1, 1, 1]), atol=1e-15)
    for mu in range(4):
        np.testing.assert_allclose(g5 @ g[mu] + g[mu] @ g5, 0, atol=1e-15)


# ---------------------------------------------------------------- adjoint links

def test_adjoint_link_closed_form_and_group_properties():
    q = synth.haar_quaternions(20, synth.Rng(3))
    for k in range(10):
        R = oracle.adjoint_link(q[k])
        np.testing.assert_allclose(R, dr.rotation(q[k]), atol=1e-14)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        R2 = oracle.adjoint_link(q[k + 10])
        R12 = oracle.adjoint_link(synth.quat_mul(q[k], q[k + 10]))
        np.testing.assert_allclose(R12, R @ R2, atol=1e-14)
    # -1 in SU(2) maps to the identity rotation
    np.testing.assert_allclose(oracle.adjoint_link(np.array([-1.0, 0, 0, 0])), np.eye(3), atol=0)


def test_expanded_fundamental_links_are_su2():
    d = (2, 2, 2, 2)
    q = synth.haar_links(d, 4)
    L = oracle.expand_links(d, 2, q)
    for mu in range(4):
        for x in range(4):
            np.testing.assert_allclose(L[mu, x], dr.su2(q[mu, x]), atol=1e-15)
            np.testing.assert_allclose(L[mu, x] @ L[mu, x].conj().T, np.eye(2), atol=1e-14)
            assert abs(np.linalg.det(L[mu, x]) - 1) < 1e-14


# ---------------------------------------------------------------- closed forms

def free_field_symbol(p, m0):
    s = (m0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        s = s + 1j * np.sin(p[mu]) * dr.GAMMA[mu]
    return s


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8), (6, 2, 4, 2)])
def test_free_field_plane_wave(nc, dims):
    V = int(np.prod(dims))
    L = oracle.expand_links(dims, nc, synth.identity_links(dims))
    x = coords(dims)
    m0 = 0.1
    for trial in range(3):
        n = np.array([RNG.integers(0, d) for d in dims])
        p = 2 * np.pi * n / np.array(dims)
        u = RNG.normal(size=(4, nc)) + 1j * RNG.normal(size=(4, nc))
        phase = np.exp(1j * (x @ p))
        psi = phase[:, None, None] * u[None]
        want = phase[:, None, None] * (free_field_symbol(p, m0) @ u)[None]
        got = oracle.dirac(dims, L, m0, psi)
        assert rel(got, want) < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_flat_connection(nc):
    """U_mu(x) = g for all x, mu: colour eigenvectors of the link see p -> p + theta."""
    dims = (4, 6, 4, 2)
    g = synth.haar_quaternions(1, synth.Rng(11))[0]
    q = np.broadcast_to(g, (4, int(np.prod(dims)), 4)).copy()
    L = oracle.expand_links(dims, nc, q)
    M = dr.su2(g) if nc == 2 else dr.rotation(g)
    evals, evecs = np.linalg.eig(M)
    x = coords(dims)
    m0 = -0.3
    for k in range(nc):
        theta = np.angle(evals[k])
        v = evecs[:, k]
        n = np.array([1, 2, 3, 1])
        p = 2 * np.pi * n / np.array(dims)
        s = RNG.normal(size=4) + 1j * RNG.normal(size=4)
        phase = np.exp(1j * (x @ p))
        psi = phase[:, None, None] * np.einsum("s,c->sc", s, v)[None]
        want = phase[:, None, None] * np.einsum("s,c->sc", free_field_symbol(p + theta, m0) @ s, v)[None]
        got = oracle.dirac(dims, L, m0, psi)
        assert rel(got, want) < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_antiperiodic_links_in_time(nc):
    """U_0 = -1, U_k = 1: the fundamental sees p_0 -> p_0 + pi, the adjoint sees nothing."""
    dims = (4, 4, 2, 2)
    V = int(np.prod(dims))
    q = synth.identity_links(dims)
    q[0, :, 0] = -1.0
    L = oracle.expand_links(dims, nc, q)
    x = coords(dims)
    n = np.array([1, 1, 0, 1])
    p = 2 * np.pi * n / np.array(dims)
    u = RNG.normal(size=(4, nc)) + 1j * RNG.normal(size=(4, nc))
    phase = np.exp(1j * (x @ p))
    psi = phase[:, None, None] * u[None]
    shift = np.array([np.pi, 0, 0, 0]) if nc == 2 else np.zeros(4)
    want = phase[:, None, None] * (free_field_symbol(p + shift, 0.2) @ u)[None]
    assert rel(oracle.dirac(dims, L, 0.2, psi), want) < 1e-14
    assert V == 64


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [1, 5, 8, 15])
def test_free_field_antiperiodic_plane_wave(nc, bc):
    """Antiperiodic in direction mu: the momenta are p_mu = (2n+1) pi / L_mu,
    and e^{ipx} u restricted to the box is an eigenvector with the free symbol."""
    dims = (4, 6, 2, 4)
    L = oracle.expand_links(dims, nc, synth.identity_links(dims))
    x = coords(dims)
    m0 = -0.1
    anti = np.array([(bc >> mu) & 1 for mu in range(4)])
    for trial in range(3):
        n = np.array([RNG.integers(0, d) for d in dims])
        p = (2 * n + anti) * np.pi / np.array(dims)
        u = RNG.normal(size=(4, nc)) + 1j * RNG.normal(size=(4, nc))
        phase = np.exp(1j * (x @ p))
        psi = phase[:, None, None] * u[None]
        want = phase[:, None, None] * (free_field_symbol(p, m0) @ u)[None]
        assert rel(oracle.dirac(dims, L, m0, psi, bc=bc), want) < 1e-14
        # the periodic operator does not have this eigenvector
        assert rel(oracle.dirac(dims, L, m0, psi), want) > 1e-3


def test_antiperiodic_fundamental_equals_negated_boundary_links():
    """For SU(2) fundamental fermions -1 is a gauge link: the antiperiodic operator
    is the periodic one with the links U_mu(x), x_mu = L_mu - 1, negated.  The
    adjoint representation is blind to that sign (R(-U) = R(U))."""
    dims = (4, 2, 4, 6)
    q = synth.haar_links(dims, 131)
    x = coords(dims)
    for bc in (1, 6, 15):
        qn = q.copy()
        for mu in range(4):
            if (bc >> mu) & 1:
                qn[mu, x[:, mu] == dims[mu] - 1] *= -1.0
        for nc in (2, 3):
            psi = synth.gaussian_spinor(dims, nc, 132)
            got = oracle.dirac(dims, oracle.expand_links(dims, nc, q), 0.2, psi, bc=bc)
            neg = oracle.dirac(dims, oracle.expand_links(dims, nc, qn), 0.2, psi)
            if nc == 2:
                assert rel(got, neg) < 1e-15
            else:
                per = oracle.dirac(dims, oracle.expand_links(dims, nc, q), 0.2, psi)
                assert rel(neg, per) < 1e-15 and rel(got, per) > 1e-2


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [0, 15])
def test_gamma5_hermiticity(nc, bc):
    dims = (4, 2, 4, 6)
    q = synth.haar_links(dims, 21)
    L = oracle.expand_links(dims, nc, q)
    phi = synth.gaussian_spinor(dims, nc, 22)
    psi = synth.gaussian_spinor(dims, nc, 23)
    m0 = 0.05
    lhs = inner(phi, oracle.dirac(dims, L, m0, psi, bc=bc))
    rhs = inner(oracle.gamma5(oracle.dirac(dims, L, m0, oracle.gamma5(phi), bc=bc)), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    # the even-odd Schur operator and its stated adjoint
    even = oracle.parity_mask(dims) == 0
    phi[~even] = 0
    psi[~even] = 0
    lhs = inner(phi, oracle.schur(dims, L, m0, psi, bc=bc))
    rhs = inner(oracle.schur(dims, L, m0, phi, dagger=True, bc=bc), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_gauge_covariance(nc):
    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    q = synth.haar_links(dims, 31)
    g = synth.haar_quaternions(V, synth.Rng(32))
    idx = np.arange(V).reshape(dims)
    qg = np.empty_like(q)
    for mu in range(4):
        fwd = np.roll(idx, -1, axis=mu).reshape(-1)
        qg[mu] = synth.quat_mul(synth.quat_mul(g, q[mu]), synth.quat_conj(g[fwd]))
    G = np.array([dr.su2(gx) if nc == 2 else dr.rotation(gx) for gx in g])
    psi = synth.gaussian_spinor(dims, nc, 33)
    psig = np.einsum("xcd,xsd->xsc", G, psi)
    m0 = 0.3
    lhs = oracle.dirac(dims, oracle.expand_links(dims, nc, qg), m0, psig)
    rhs = np.einsum("xcd,xsd->xsc", G, oracle.dirac(dims, oracle.expand_links(dims, nc, q), m0, psi))
    assert rel(lhs, rhs) < 1e-14


# ---------------------------------------------------------------- dense brute force

@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 4)])
@pytest.mark.parametrize("bc", [0, 1, 10, 15])
def test_dense_bruteforce_full_operator(nc, dims, bc):
    q = synth.haar_links(dims, 41)
    L = oracle.expand_links(dims, nc, q)
    D = dr.dirac_dense(dims, q, nc, 0.1, bc)
    for seed in (42, 43):
        psi = synth.gaussian_spinor(dims, nc, seed)
        assert rel(oracle.dirac(dims, L, 0.1, psi, bc=bc).reshape(-1), D @ psi.reshape(-1)) < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [0, 9])
def test_dense_schur_complement(nc, bc):
    dims = (2, 4, 2, 2)
    m0 = -0.2
    q = synth.haar_links(dims, 51)
    L = oracle.expand_links(dims, nc, q)
    D = dr.dirac_dense(dims, q, nc, m0, bc)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, nc, D)
    np.testing.assert_allclose(Dee, (4 + m0) * np.eye(len(e)), atol=0)
    np.testing.assert_allclose(Doo, (4 + m0) * np.eye(len(o)), atol=0)
    Mhat = Dee - Deo @ np.linalg.solve(Doo, Doe)
    # det D = det(D_oo) det(Mhat)
    s1, l1 = np.linalg.slogdet(D)
    s2, l2 = np.linalg.slogdet(Doo)
    s3, l3 = np.linalg.slogdet(Mhat)
    assert abs(l1 - (l2 + l3)) < 1e-10 and abs(s1 - s2 * s3) < 1e-10
    psi = synth.gaussian_spinor(dims, nc, 52)
    psi[oracle.parity_mask(dims) == 1] = 0
    flat = psi.reshape(-1)
    got = oracle.schur(dims, L, m0, psi, bc=bc).reshape(-1)
    assert rel(got[e], Mhat @ flat[e]) < 1e-14
    assert np.all(got[o] == 0)
    gotd = oracle.schur(dims, L, m0, psi, dagger=True, bc=bc).reshape(-1)
    assert rel(gotd[e], Mhat.conj().T @ flat[e]) < 1e-14
    gotn = oracle.normal(dims, L, m0, psi, bc=bc).reshape(-1)
    assert rel(gotn[e], Mhat.conj().T @ (Mhat @ flat[e])) < 1e-14


def test_hop_sites_matches_parity_hop():
    dims = (4, 4, 4, 6)
    q = synth.haar_links(dims, 61)
    for nc in (2, 3):
        L = oracle.expand_links(dims, nc, q)
        psi = synth.gaussian_spinor(dims, nc, 62)
        full = oracle.hop(dims, L, psi)
        for par in (0, 1):
            h = oracle.hop(dims, L, psi, parity=par)
            mask = oracle.parity_mask(dims) == par
            np.testing.assert_array_equal(h[mask], full[mask])
            assert np.all(h[~mask] == 0)
        sites = RNG.choice(int(np.prod(dims)), size=17, replace=False)
        np.testing.assert_array_equal(oracle.hop_sites(dims, L, psi, sites), full[sites])


# ---------------------------------------------------------------- solvers

@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [0, 1])
def test_cg_against_dense_solve(nc, bc):
    dims = (2, 4, 2, 4)
    m0 = -0.2
    q = synth.haar_links(dims, 71)
    L = oracle.expand_links(dims, nc, q)
    D = dr.dirac_dense(dims, q, nc, m0, bc)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, nc, D)
    Mhat = Dee - Deo @ np.linalg.solve(Doo, Doe)
    A = Mhat.conj().T @ Mhat
    assert np.linalg.eigvalsh(A).min() > 0
    b = synth.gaussian_spinor(dims, nc, 72)
    b[oracle.parity_mask(dims) == 1] = 0
    x, iters, true_rel, ok = oracle.cg(dims, L, m0, b, tol=1e-12, bc=bc)
    assert ok and true_rel <= 1e-12
    xd = np.linalg.solve(A, b.reshape(-1)[e])
    assert rel(x.reshape(-1)[e], xd) < 1e-10
    assert np.all(x.reshape(-1)[o] == 0)
    # ||b - A x|| recomputed densely
    assert np.linalg.norm(b.reshape(-1)[e] - A @ x.reshape(-1)[e]) / np.linalg.norm(b) < 1e-11


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("bc", [0, 1])
def test_eo_solve_of_full_operator(nc, bc):
    """Source preparation + Schur solve + odd reconstruction solves D x = b."""
    dims = (4, 2, 2, 4)
    m0 = 0.1
    q = synth.haar_links(dims, 81)
    L = oracle.expand_links(dims, nc, q)
    b = synth.gaussian_spinor(dims, nc, 82)
    bhat = oracle.eo_source(dims, L, m0, b, bc=bc)
    # solve Mhat x_e = bhat via CG on Mhat^+ Mhat x_e = Mhat^+ bhat
    rhs = oracle.schur(dims, L, m0, bhat, dagger=True, bc=bc)
    xe, it, tr, ok = oracle.cg(dims, L, m0, rhs, tol=1e-13, bc=bc)
    assert ok
    x = oracle.eo_reconstruct(dims, L, m0, b, xe, bc=bc)
    assert rel(oracle.dirac(dims, L, m0, x, bc=bc), b) < 1e-11
    D = dr.dirac_dense(dims, q, nc, m0, bc)
    assert rel(x.reshape(-1), np.linalg.solve(D, b.reshape(-1))) < 1e-10


# ---------------------------------------------------------------- link derivatives

def _su2_exp(w):
    """exp(i w.s / 2) as a quaternion."""
    th = np.linalg.norm(w) / 2
    n = w / np.linalg.norm(w)
    return np.concatenate([[np.cos(th)], np.sin(th) * n])


@pytest.mark.parametrize("bc", [0, 5])
def test_link_grad_matches_finite_differences(bc):
    dims = (2, 4, 2, 2)
    V = int(np.prod(dims))
    q = synth.haar_links(dims, 91)
    a = synth.gaussian_spinor(dims, 2, 92)
    b = synth.gaussian_spinor(dims, 2, 93)
    G = oracle.link_grad(dims, a, b, bc=bc)

    def f(qq):
        # the operator itself from the independent dense build
        return inner(a.reshape(-1), dr.hopping_dense(dims, qq, 2, bc) @ b.reshape(-1)).real

    eps = 1e-6
    for _ in range(12):
        mu, x, k = RNG.integers(4), RNG.integers(V), RNG.integers(4)
        qp, qm = q.copy(), q.copy()
        qp[mu, x, k] += eps
        qm[mu, x, k] -= eps
        fd = (f(qp) - f(qm)) / (2 * eps)  # f is linear in q: exact up to rounding
        assert abs(fd - G[mu, x, k]) < 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("bc", [0, 3])
def test_force_matches_finite_differences_of_solve_loss(bc):
    """S = Re<eta, (Mhat^+ Mhat)^-1 eta>; F = dS/dw under U -> exp(i w.s/2) U.

    dS = 2c Re[<Y, dH_eo H_oe X> + <H_eo^+ Y, dH_oe X>],  X = A^-1 eta,
    Y = Mhat X, c = 1/(4(4+m0)), H_eo^+ = g5 H_oe g5; i.e. 2c times the
    derivative of Re<a, H b> with a = (Y, g5 H_oe g5 Y), b = (X, H_oe X).
    S itself is evaluated with dense solves (independent of the oracle).
    """
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0 = 0.2
    A4 = 4 + m0
    q = synth.haar_links(dims, 101)
    L = oracle.expand_links(dims, 2, q)
    eta = synth.gaussian_spinor(dims, 2, 102)
    even = oracle.parity_mask(dims) == 0
    eta[~even] = 0

    def S(qq):
        D = dr.dirac_dense(dims, qq, 2, m0, bc)
        Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
        M = Dee - Deo @ np.linalg.solve(Doo, Doe)
        y = eta.reshape(-1)[e]
        return np.vdot(y, np.linalg.solve(M.conj().T @ M, y)).real

    X, it, tr, ok = oracle.cg(dims, L, m0, eta, tol=1e-14, maxiter=5000, bc=bc)
    Y = oracle.schur(dims, L, m0, X, bc=bc)
    Z = oracle.hop(dims, L, X, parity=1, bc=bc)                        # H_oe X on odd sites
    W = oracle.gamma5(oracle.hop(dims, L, oracle.gamma5(Y), parity=1, bc=bc))  # H_eo^+ Y on odd sites
    a = np.where(even[:, None, None], Y, W)
    b = np.where(even[:, None, None], X, Z)
    F = 2.0 / (4.0 * A4) * oracle.force(dims, L, a, b, bc=bc)
    eps = 1e-5
    for _ in range(10):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        w /= np.linalg.norm(w)
        qp, qm = q.copy(), q.copy()
        qp[mu, x] = synth.quat_mul(_su2_exp(eps * w), q[mu, x])
        qm[mu, x] = synth.quat_mul(_su2_exp(-eps * w), q[mu, x])
        fd = (S(qp) - S(qm)) / (2 * eps)
        an = F[mu, x] @ w
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


# ---------------------------------------------------------------- plaquette

def test_plaquette():
    dims = (4, 4, 2, 2)
    assert abs(oracle.plaquette(dims, synth.identity_links(dims)) - 1) < 1e-15
    q = synth.haar_links(dims, 111)
    p = oracle.plaquette(dims, q)
    assert abs(p - synth.mean_plaquette(q, dims)) < 1e-14
    # gauge invariance
    V = int(np.prod(dims))
    g = synth.haar_quaternions(V, synth.Rng(112))
    idx = np.arange(V).reshape(dims)
    qg = np.empty_like(q)
    for mu in range(4):
        fwd = np.roll(idx, -1, axis=mu).reshape(-1)
        qg[mu] = synth.quat_mul(synth.quat_mul(g, q[mu]), synth.quat_conj(g[fwd]))
    assert abs(oracle.plaquette(dims, qg) - p) < 1e-14


def test_smeared_field_reaches_target_plaquette():
    dims = (4, 4, 4, 4)
    q = synth.haar_links(dims, 121)
    qs, steps, p = synth.ape_smear_to_plaquette(q, dims, target=0.6)
    assert steps >= 1
    assert abs(oracle.plaquette(dims, qs) - 0.6) < 2e-3
    np.testing.assert_allclose(np.linalg.norm(qs, axis=-1), 1.0, atol=1e-14)
