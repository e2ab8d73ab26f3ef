"""Pins of the oracle's clover-term HMC force (oracle/clover.py: clover_derivative,
CloverFermions).

The paper (arXiv:2411.18511, Sec. 2.2) measures the clover operator and names
the HMC as its consumer without writing the force down.  The oracle's analytic
derivatives are tied to facts that do not come from them:

* clover_derivative against central finite differences of Re sum tr[C Lam] for
  a random insertion Lam, C from the site-term code (itself pinned by closed
  forms and a dense build in tests/test_oracle_clover.py);
* the whole two-flavour force (pseudofermion and det A_oo) against central
  finite differences of S = Re<eta, (Mhat^+ Mhat)^-1 eta> - 2 sum_odd log det A,
  both evaluated with dense matrices from tests/dense_ref.py;
* the heat-bath normalisation S_pf = |xi|^2 for eta = Mhat^+ xi;
* the exponential form: exp_insertion (the divided differences of exp in the
  eigenbasis of A) against finite differences of Re sum tr[A_exp Lam], and its
  whole force against dense-matrix actions built with scipy's expm.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import clover as ocl
from oracle import hmc
from tests import dense_ref as dr

RNG = np.random.default_rng(4242)


def exp_update(q, mu, x, w, eps):
    out = q.copy()
    out[mu, x] = hmc.link_update(q[mu, x][None], w[None], eps)[0]
    return out


def smeared(dims, seed):
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, seed), dims, 0.6)
    return q


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 2, 4, 2)])
def test_clover_derivative_matches_finite_differences(dims):
    V = int(np.prod(dims))
    q = synth.haar_links(dims, 501)
    Lam = RNG.normal(size=(V, 8, 8)) + 1j * RNG.normal(size=(V, 8, 8))

    def f(qq):
        C = ocl.clover_generator(dims, oracle.expand_links(dims, 2, qq))
        return float(np.real(np.einsum("xij,xji->", C, Lam)))

    G = ocl.clover_derivative(dims, oracle.expand_links(dims, 2, q), Lam)
    eps = 1e-5
    for _ in range(16):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (f(exp_update(q, mu, x, w, eps)) - f(exp_update(q, mu, x, w, -eps))) / (2 * eps)
        assert abs(fd - G[mu, x] @ w) <= 1e-7 * max(1.0, abs(fd)), (mu, x, fd, G[mu, x] @ w)


def _dense_action(dims, q, m0, csw, eta, bc):
    A = dr.clover_site_dense(dims, q, 2, m0, csw)
    D = dr.dirac_clover_dense(dims, q, 2, A, bc)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
    M = Dee - Deo @ np.linalg.solve(Doo, Doe)
    y = eta.reshape(-1)[e]
    S_pf = np.vdot(y, np.linalg.solve(M.conj().T @ M, y)).real
    odd = oracle.parity_mask(dims) == 1
    S_det = -2.0 * sum(np.linalg.slogdet(A[k])[1] for k in np.where(odd)[0])
    return S_pf + S_det, M, e


@pytest.mark.parametrize("bc", [0, 1])
def test_clover_fermion_force_matches_finite_differences(bc):
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0, csw = 0.1, 1.3
    q = smeared(dims, 511)
    eta = synth.gaussian_spinor(dims, 2, 512)
    eta[oracle.parity_mask(dims) == 1] = 0
    ferm = ocl.CloverFermions(dims, m0, csw, eta, bc=bc, tol=1e-14)
    S0, _, _ = _dense_action(dims, q, m0, csw, eta, bc)
    assert abs(ferm.action(q) - S0) <= 1e-10 * abs(S0)
    F = ferm.force(q)
    eps = 1e-5
    for _ in range(12):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (_dense_action(dims, exp_update(q, mu, x, w, eps), m0, csw, eta, bc)[0]
              - _dense_action(dims, exp_update(q, mu, x, w, -eps), m0, csw, eta, bc)[0]) / (2 * eps)
        assert abs(fd - F[mu, x] @ w) <= 1e-6 * max(1.0, abs(fd)), (mu, x, fd, F[mu, x] @ w)


def test_clover_heat_bath_normalisation():
    dims = (2, 2, 2, 4)
    m0, csw = 0.1, 1.0
    q = smeared(dims, 521)
    _, M, e = _dense_action(dims, q, m0, csw, np.zeros((int(np.prod(dims)), 4, 2), complex), 0)
    xi = (RNG.normal(size=len(e)) + 1j * RNG.normal(size=len(e))) / np.sqrt(2)
    eta = np.zeros(int(np.prod(dims)) * 8, dtype=complex)
    eta[e] = M.conj().T @ xi
    eta = eta.reshape(-1, 4, 2)
    ferm = ocl.CloverFermions(dims, m0, csw, eta, tol=1e-14)
    L, A, x = ferm.solve(q)
    assert abs(np.vdot(eta, x).real - np.vdot(xi, xi).real) <= 1e-10 * np.vdot(xi, xi).real


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.OMELYAN])
def test_clover_trajectory_reversible_and_second_order(integrator):
    dims = (4, 2, 2, 2)
    m0, csw = 0.1, 1.0
    q = smeared(dims, 531)
    p = np.random.default_rng(532).normal(size=(4, int(np.prod(dims)), 3))
    eta = synth.gaussian_spinor(dims, 2, 533) / np.sqrt(2.0)
    eta[oracle.parity_mask(dims) == 1] = 0
    ferm = ocl.CloverFermions(dims, m0, csw, eta, bc=1)
    q1, p1, i1 = hmc.trajectory(dims, q, p, 2.2, 3, 0.3, integrator, ferm)
    q2, p2, i2 = hmc.trajectory(dims, q1, -p1, 2.2, 3, 0.3, integrator, ferm)
    assert np.abs(q2 - q).max() < 1e-10 and np.abs(p2 + p).max() < 1e-9
    dh = [abs(hmc.trajectory(dims, q, p, 2.2, n, 0.5, integrator, ferm)[2]["dH"]) for n in (8, 16)]
    assert 3.8 < dh[0] / dh[1] < 4.2, dh


# ---------------------------------------------------------------- exponential clover

def test_exp_insertion_matches_finite_differences():
    """d Re sum tr[A_exp Lam] = c_sw Re sum tr[dC Lam'] with Lam' from exp_insertion:
    against central finite differences of the exponential site term."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0, csw = 0.1, 1.4
    q = synth.haar_links(dims, 541)
    Lam = RNG.normal(size=(V, 8, 8)) + 1j * RNG.normal(size=(V, 8, 8))

    def f(qq):
        A = ocl.site_term(dims, oracle.expand_links(dims, 2, qq), m0, csw, ocl.KIND_EXP)
        return float(np.real(np.einsum("xij,xji->", A, Lam)))

    L = oracle.expand_links(dims, 2, q)
    A = ocl.site_term(dims, L, m0, csw, ocl.KIND_EXP)
    G = csw * ocl.clover_derivative(dims, L, ocl.exp_insertion(A, Lam, m0))
    eps = 1e-5
    for _ in range(12):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (f(exp_update(q, mu, x, w, eps)) - f(exp_update(q, mu, x, w, -eps))) / (2 * eps)
        assert abs(fd - G[mu, x] @ w) <= 1e-7 * max(1.0, abs(fd)), (mu, x, fd, G[mu, x] @ w)


def _dense_action_exp(dims, q, m0, csw, eta, bc):
    A = dr.clover_site_dense(dims, q, 2, m0, csw, exponential=True)
    D = dr.dirac_clover_dense(dims, q, 2, A, bc)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
    M = Dee - Deo @ np.linalg.solve(Doo, Doe)
    y = eta.reshape(-1)[e]
    odd = oracle.parity_mask(dims) == 1
    S_det = -2.0 * sum(np.linalg.slogdet(A[k])[1] for k in np.where(odd)[0])
    return np.vdot(y, np.linalg.solve(M.conj().T @ M, y)).real + S_det


def test_exp_clover_fermion_force_matches_finite_differences():
    """The exponential form's whole force (its det A_oo is constant) against dense-matrix actions."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0, csw, bc = 0.1, 1.3, 1
    q = smeared(dims, 551)
    eta = synth.gaussian_spinor(dims, 2, 552)
    eta[oracle.parity_mask(dims) == 1] = 0
    ferm = ocl.CloverFermions(dims, m0, csw, eta, bc=bc, tol=1e-14, kind=ocl.KIND_EXP)
    S0 = _dense_action_exp(dims, q, m0, csw, eta, bc)
    assert abs(ferm.action(q) - S0) <= 1e-10 * abs(S0)
    F = ferm.force(q)
    eps = 1e-5
    for _ in range(12):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (_dense_action_exp(dims, exp_update(q, mu, x, w, eps), m0, csw, eta, bc)
              - _dense_action_exp(dims, exp_update(q, mu, x, w, -eps), m0, csw, eta, bc)) / (2 * eps)
        assert abs(fd - F[mu, x] @ w) <= 1e-6 * max(1.0, abs(fd)), (mu, x, fd, F[mu, x] @ w)


@pytest.mark.parametrize("kind", [ocl.KIND_SW, ocl.KIND_EXP])
def test_clover_hasenbusch_force_matches_finite_differences(kind):
    """Clover fermions with Hasenbusch's two pseudofermions: S = Re<eta, (Mhat_H^+ Mhat_H)^-1 eta>
    + Re<eta2, (Mhat^+ Mhat)^-1 eta2> - 2 sum_odd log det A, eta2 = Mhat_H^+ phi, all from dense
    matrices; the oracle's force against its central finite differences."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0, mh, csw, bc = 0.05, 0.5, 1.2, 1
    q = smeared(dims, 561)
    eta = synth.gaussian_spinor(dims, 2, 562)
    phi = synth.gaussian_spinor(dims, 2, 563)
    odd = oracle.parity_mask(dims) == 1
    eta[odd] = 0
    phi[odd] = 0
    exponential = kind == ocl.KIND_EXP

    def S(qq):
        def schur_dense(m):
            A = dr.clover_site_dense(dims, qq, 2, m, csw, exponential=exponential)
            D = dr.dirac_clover_dense(dims, qq, 2, A, bc)
            Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
            return Dee - Deo @ np.linalg.solve(Doo, Doe), e, A

        M, e, A = schur_dense(m0)
        MH, _, _ = schur_dense(mh)
        y1 = eta.reshape(-1)[e]
        y2 = MH.conj().T @ phi.reshape(-1)[e]
        S_det = -2.0 * sum(np.linalg.slogdet(A[k])[1] for k in np.where(odd)[0])
        return (np.vdot(y1, np.linalg.solve(MH.conj().T @ MH, y1)).real
                + np.vdot(y2, np.linalg.solve(M.conj().T @ M, y2)).real + S_det)

    ferm = ocl.CloverHasenbusch(dims, m0, mh, csw, eta, phi, bc=bc, tol=1e-14, kind=kind)
    S0 = S(q)
    assert abs(ferm.action(q) - S0) <= 1e-10 * abs(S0)
    F = ferm.force(q)
    eps = 1e-5
    for _ in range(10):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (S(exp_update(q, mu, x, w, eps)) - S(exp_update(q, mu, x, w, -eps))) / (2 * eps)
        assert abs(fd - F[mu, x] @ w) <= 1e-6 * max(1.0, abs(fd)), (mu, x, fd, F[mu, x] @ w)
