"""Pins of the oracle's clover and exponential-clover site terms (oracle/clover.py).

The paper (arXiv:2411.18511, Sec. 2.2) names both improvements without a
formula or an example; the oracle takes the textbook definitions, and these
tests tie it to facts that do not come from it:

* a constant abelian field on the torus (every 01-plaquette equal to
  exp(i B s_3), B T L1 a multiple of 2 pi): F_01 = i sin(B) s_3 on every site,
  so the site term's spectrum is (4+m0) +- c_sw sin(B)/2 in the fundamental
  and (4+m0) +- c_sw sin(2B)/2, (4+m0) in the adjoint (exponential clover:
  (4+m0) exp(+- c_sw sin / (2 (4+m0))));
* the free field (A = 4 + m0, D = Wilson);
* Hermiticity, chirality ([A, g5] = 0) and gauge covariance;
* an independent dense build with explicit per-site loops (tests/dense_ref.py),
  including the even-odd Schur complement, the CG and the even-odd solve.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import clover as ocl
from tests import dense_ref as dr

KINDS = [ocl.KIND_SW, ocl.KIND_EXP]


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def abelian_field(dims, n=1):
    """U_1(x) = exp(i s_3 B x0); U_0 = exp(-i s_3 B T x1) on the last time slice, 1 elsewhere;
    U_2 = U_3 = 1.  B = 2 pi n / (T L1): every 01-plaquette is exp(i s_3 B)."""
    T, L1 = dims[0], dims[1]
    B = 2 * np.pi * n / (T * L1)
    x = np.indices(dims).reshape(4, -1).T
    q = synth.identity_links(dims)

    def rot3(theta):
        out = np.zeros((len(theta), 4))
        out[:, 0] = np.cos(theta)
        out[:, 3] = np.sin(theta)
        return out

    q[1] = rot3(B * x[:, 0])
    last = x[:, 0] == T - 1
    q[0, last] = rot3(-B * T * x[last, 1])
    return q, B


def test_sigma_matrices():
    g5 = oracle.gamma(4)
    for mu in range(4):
        for nu in range(4):
            s = ocl.sigma(mu, nu)
            np.testing.assert_allclose(s, s.conj().T, atol=1e-15)
            np.testing.assert_allclose(s, -ocl.sigma(nu, mu), atol=1e-15)
            np.testing.assert_allclose(s @ g5, g5 @ s, atol=1e-15)
            if mu != nu:
                np.testing.assert_allclose(s @ s, np.eye(4), atol=1e-15)
            np.testing.assert_allclose(s, dr.sigma_dense(mu, nu), atol=1e-15)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nc", [2, 3])
def test_constant_abelian_field_closed_form(nc, kind):
    dims = (4, 4, 2, 2)
    q, B = abelian_field(dims)
    assert abs(oracle.plaquette(dims, q) - (5 + np.cos(B)) / 6) < 1e-14  # 1 of the 6 planes carries B
    L = oracle.expand_links(dims, nc, q)
    F = ocl.field_strength(dims, L)
    m0, csw = -0.3, 1.7
    a = 4 + m0
    if nc == 2:
        s3 = np.diag([1.0, -1.0])
        np.testing.assert_allclose(F[0, 1], np.broadcast_to(1j * np.sin(B) * s3, F[0, 1].shape), atol=1e-15)
        lam = np.sin(B) / 2 * np.array([-1, 1])
        mult = [4, 4]
    else:
        lam = np.sin(2 * B) / 2 * np.array([-1, 0, 1])
        mult = [4, 4, 4]
    for mu in range(4):
        for nu in range(4):
            if {mu, nu} != {0, 1}:
                assert np.abs(F[mu, nu]).max() < 1e-15
    c = np.repeat(lam, mult)
    want = np.sort(a + csw * c) if kind == ocl.KIND_SW else np.sort(a * np.exp(csw * c / a))
    A = ocl.site_term(dims, L, m0, csw, kind)
    for x in range(A.shape[0]):
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A[x])), want, atol=1e-14)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nc", [2, 3])
def test_free_field_reduces_to_wilson(nc, kind):
    dims = (4, 2, 4, 2)
    L = oracle.expand_links(dims, nc, synth.identity_links(dims))
    A = ocl.site_term(dims, L, 0.1, 1.9, kind)
    np.testing.assert_allclose(A, np.broadcast_to(4.1 * np.eye(4 * nc), A.shape), atol=1e-15)
    psi = synth.gaussian_spinor(dims, nc, 7)
    assert rel(ocl.dirac(dims, L, A, psi), oracle.dirac(dims, L, 0.1, psi)) < 1e-15


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nc", [2, 3])
def test_site_term_hermitian_and_chiral(nc, kind):
    dims = (4, 2, 2, 4)
    L = oracle.expand_links(dims, nc, synth.haar_links(dims, 201))
    A = ocl.site_term(dims, L, -0.2, 1.3, kind)
    np.testing.assert_allclose(A, np.conj(np.swapaxes(A, 1, 2)), atol=1e-14)
    G5 = np.kron(oracle.gamma(4), np.eye(nc))
    np.testing.assert_allclose(np.einsum("ij,xjk->xik", G5, A), np.einsum("xij,jk->xik", A, G5), atol=1e-14)
    assert np.abs(A - (4 - 0.2) * np.eye(4 * nc)).max() > 0.1  # a genuinely non-trivial term


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nc", [2, 3])
def test_gauge_covariance(nc, kind):
    dims = (4, 4, 2, 2)
    V = int(np.prod(dims))
    q = synth.haar_links(dims, 211)
    g = synth.haar_quaternions(V, synth.Rng(212))
    idx = np.arange(V).reshape(dims)
    qg = np.empty_like(q)
    for mu in range(4):
        fwd = np.roll(idx, -1, axis=mu).reshape(-1)
        qg[mu] = synth.quat_mul(synth.quat_mul(g, q[mu]), synth.quat_conj(g[fwd]))
    G = np.array([dr.su2(gx) if nc == 2 else dr.rotation(gx) for gx in g])
    psi = synth.gaussian_spinor(dims, nc, 213)
    psig = np.einsum("xcd,xsd->xsc", G, psi)
    L, Lg = oracle.expand_links(dims, nc, q), oracle.expand_links(dims, nc, qg)
    A, Ag = ocl.site_term(dims, L, 0.2, 1.5, kind), ocl.site_term(dims, Lg, 0.2, 1.5, kind)
    lhs = ocl.dirac(dims, Lg, Ag, psig)
    rhs = np.einsum("xcd,xsd->xsc", G, ocl.dirac(dims, L, A, psi))
    assert rel(lhs, rhs) < 1e-14


@pytest.mark.parametrize("bc", [0, 9])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nc", [2, 3])
def test_dense_build(nc, kind, bc):
    dims = (2, 4, 2, 4)
    q = synth.haar_links(dims, 221)
    L = oracle.expand_links(dims, nc, q)
    m0, csw = -0.1, 1.4
    A = ocl.site_term(dims, L, m0, csw, kind)
    Ad = dr.clover_site_dense(dims, q, nc, m0, csw, exponential=kind == ocl.KIND_EXP)
    np.testing.assert_allclose(A, Ad, atol=1e-14)
    D = dr.dirac_clover_dense(dims, q, nc, Ad, bc)
    psi = synth.gaussian_spinor(dims, nc, 222)
    assert rel(ocl.dirac(dims, L, A, psi, bc=bc).reshape(-1), D @ psi.reshape(-1)) < 1e-14


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nc", [2, 3])
def test_dense_schur_cg_and_eo_solve(nc, kind):
    dims = (2, 4, 2, 4)
    bc = 1
    q = synth.haar_links(dims, 231)
    L = oracle.expand_links(dims, nc, q)
    m0, csw = 0.1, 1.2
    A = ocl.site_term(dims, L, m0, csw, kind)
    D = dr.dirac_clover_dense(dims, q, nc, dr.clover_site_dense(dims, q, nc, m0, csw, kind == ocl.KIND_EXP), bc)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, nc, D)
    Mhat = Dee - Deo @ np.linalg.solve(Doo, Doe)
    psi = synth.gaussian_spinor(dims, nc, 232)
    psi[oracle.parity_mask(dims) == 1] = 0
    flat = psi.reshape(-1)
    got = ocl.schur(dims, L, A, psi, bc=bc).reshape(-1)
    assert rel(got[e], Mhat @ flat[e]) < 1e-14 and np.all(got[o] == 0)
    gotd = ocl.schur(dims, L, A, psi, dagger=True, bc=bc).reshape(-1)
    assert rel(gotd[e], Mhat.conj().T @ flat[e]) < 1e-14
    # CG on Mhat^+ Mhat, and the even-odd solve of D x = b
    b = synth.gaussian_spinor(dims, nc, 233)
    rhs = ocl.schur(dims, L, A, ocl.eo_source(dims, L, A, b, bc=bc), dagger=True, bc=bc)
    xe, it, tr, ok = ocl.cg(dims, L, A, rhs, tol=1e-13, bc=bc)
    assert ok and tr <= 1e-13
    x = ocl.eo_reconstruct(dims, L, A, b, xe, bc=bc)
    assert rel(x.reshape(-1), np.linalg.solve(D, b.reshape(-1))) < 1e-10


def test_exponential_matches_scipy_expm():
    from scipy.linalg import expm

    dims = (2, 2, 4, 2)
    L = oracle.expand_links(dims, 2, synth.haar_links(dims, 241))
    C = ocl.clover_generator(dims, L)
    A = ocl.site_term(dims, L, -0.4, 2.0, ocl.KIND_EXP)
    for x in range(C.shape[0]):
        np.testing.assert_allclose(A[x], 3.6 * expm(2.0 * C[x] / 3.6), atol=1e-14)
