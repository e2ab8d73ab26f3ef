"""Pins of the oracle's HMC molecular dynamics (oracle/hmc.py).

The paper (arXiv:2411.18511) names HMC as the consumer of the even-odd solver
without writing it down; the oracle takes the textbook scheme, and these
tests tie it to facts that do not come from it:

* the gauge force equals central finite differences of the gauge action (the
  action itself comes from the plaquette, pinned in test_oracle_pins.py);
* the link update equals the matrix exponential (scipy.linalg.expm);
* leapfrog and Omelyan trajectories are reversible: flipping the momenta at
  the end and integrating again returns to the start;
* both are second-order integrators: halving the step size divides Delta H
  by about four;
* the fermion force is oracle.force composed as in the HMC (that composition
  is pinned against finite differences of a dense solve in test_oracle_pins.py).
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import hmc

RNG = np.random.default_rng(777)


def smeared(dims, seed):
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, seed), dims, 0.6)
    return q


def momenta(dims, seed):
    return np.random.default_rng(seed).normal(size=(4, int(np.prod(dims)), 3))


def pseudofermion(dims, m0, seed):
    """A Gaussian even-site pseudofermion field (its distribution does not
    matter to these properties of the integrator)."""
    xi = synth.gaussian_spinor(dims, 2, seed) / np.sqrt(2.0)
    xi[oracle.parity_mask(dims) == 1] = 0
    return xi


def exp_update(q, mu, x, w, eps):
    """U_mu(x) -> exp(i eps w.s/2) U_mu(x)."""
    out = q.copy()
    out[mu, x] = hmc.link_update(q[mu, x][None], w[None], eps)[0]
    return out


def test_gauge_force_matches_finite_differences():
    dims = (4, 2, 2, 4)
    V = int(np.prod(dims))
    beta = 2.3
    q = synth.haar_links(dims, 11)
    F = hmc.gauge_force(dims, q, beta)
    eps = 1e-5
    for _ in range(12):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (hmc.gauge_action(dims, exp_update(q, mu, x, w, eps), beta)
              - hmc.gauge_action(dims, exp_update(q, mu, x, w, -eps), beta)) / (2 * eps)
        assert abs(fd - F[mu, x] @ w) < 1e-7 * max(1.0, abs(fd)), (fd, F[mu, x] @ w)


def test_link_update_is_the_matrix_exponential():
    from scipy.linalg import expm

    dims = (2, 2, 2, 2)
    q = synth.haar_links(dims, 21)
    p = momenta(dims, 22)
    eps = 0.37
    qn = hmc.link_update(q, p, eps)
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    for mu in range(4):
        for x in range(0, q.shape[1], 3):
            X = 0.5j * eps * sum(p[mu, x, a] * s[a] for a in range(3))
            want = expm(X) @ hmc._su2(q[mu, x])
            np.testing.assert_allclose(hmc._su2(qn[mu, x]), want, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(qn, axis=-1), 1.0, atol=1e-14)


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.OMELYAN])
@pytest.mark.parametrize("with_fermions", [False, True])
def test_reversibility(integrator, with_fermions):
    dims = (4, 2, 2, 2) if with_fermions else (4, 4, 2, 2)
    beta, m0 = 2.2, 0.1
    q = smeared(dims, 31)
    p = momenta(dims, 32)
    ferm = hmc.Fermions(dims, m0, pseudofermion(dims, m0, 33), bc=1) if with_fermions else None
    q1, p1, i1 = hmc.trajectory(dims, q, p, beta, 4, 0.4, integrator, ferm)
    q2, p2, i2 = hmc.trajectory(dims, q1, -p1, beta, 4, 0.4, integrator, ferm)
    assert np.abs(q2 - q).max() < 1e-10
    assert np.abs(-p2 - p).max() < 1e-9
    assert abs(i1["dH"] + i2["dH"]) < 1e-9
    assert np.abs(q1 - q).max() > 1e-3  # it moved


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.OMELYAN])
@pytest.mark.parametrize("with_fermions", [False, True])
def test_delta_h_is_second_order(integrator, with_fermions):
    dims = (4, 2, 2, 2) if with_fermions else (4, 4, 4, 4)
    beta, m0 = 2.2, 0.1
    q = smeared(dims, 41)
    p = momenta(dims, 42)
    ferm = hmc.Fermions(dims, m0, pseudofermion(dims, m0, 43)) if with_fermions else None
    dh = [abs(hmc.trajectory(dims, q, p, beta, n, 0.5, integrator, ferm)[2]["dH"]) for n in (8, 16, 32)]
    assert 3.8 < dh[0] / dh[1] < 4.2 and 3.8 < dh[1] / dh[2] < 4.2, dh


def test_omelyan_error_is_far_below_leapfrog():
    """The minimum-norm scheme's leading error coefficient is an order of magnitude
    below leapfrog's (Omelyan et al.); at equal step counts Delta H is far smaller."""
    dims = (4, 4, 4, 4)
    q = smeared(dims, 51)
    p = momenta(dims, 52)
    lf = abs(hmc.trajectory(dims, q, p, 2.2, 16, 0.5, hmc.LEAPFROG)[2]["dH"])
    om = abs(hmc.trajectory(dims, q, p, 2.2, 16, 0.5, hmc.OMELYAN)[2]["dH"])
    assert om < lf / 5, (om, lf)


# ---------------------------------------------------------------- Hasenbusch

def _dense_schur(dims, q, m0, bc):
    from tests import dense_ref as dr

    D = dr.dirac_dense(dims, q, 2, m0, bc)
    Dee, Deo, Doe, Doo, e, o = dr.eo_blocks(dims, 2, D)
    return Dee - Deo @ np.linalg.solve(Doo, Doe), e


def _hasenbusch_fields(dims, q, m0, m0_h, bc, seed):
    """eta = Mhat_H^+ xi1 and phi = Mhat_H (Mhat_H^+ Mhat_H)^-1 Mhat^+ xi2 from dense matrices."""
    M, e = _dense_schur(dims, q, m0, bc)
    MH, _ = _dense_schur(dims, q, m0_h, bc)
    rng = np.random.default_rng(seed)
    n = len(e)
    xi1 = (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(2)
    xi2 = (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(2)
    V = int(np.prod(dims))
    eta = np.zeros(V * 8, dtype=complex)
    phi = np.zeros(V * 8, dtype=complex)
    eta[e] = MH.conj().T @ xi1
    phi[e] = MH @ np.linalg.solve(MH.conj().T @ MH, M.conj().T @ xi2)
    return eta.reshape(V, 4, 2), phi.reshape(V, 4, 2), xi1, xi2


def test_hasenbusch_heat_bath_and_force():
    """S = |xi1|^2 + |xi2|^2 right after the heat bath, and the force equals
    central finite differences of S evaluated with dense solves."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    m0, m0_h, bc = 0.05, 0.6, 1
    q = smeared(dims, 61)
    eta, phi, xi1, xi2 = _hasenbusch_fields(dims, q, m0, m0_h, bc, 62)
    ferm = hmc.Hasenbusch(dims, m0, m0_h, eta, phi, bc=bc)
    S0 = ferm.action(q)
    assert abs(S0 - (np.vdot(xi1, xi1).real + np.vdot(xi2, xi2).real)) < 1e-10 * S0

    def S_dense(qq):
        M, e = _dense_schur(dims, qq, m0, bc)
        MH, _ = _dense_schur(dims, qq, m0_h, bc)
        y1 = eta.reshape(-1)[e]
        y2 = MH.conj().T @ phi.reshape(-1)[e]
        return (np.vdot(y1, np.linalg.solve(MH.conj().T @ MH, y1)).real
                + np.vdot(y2, np.linalg.solve(M.conj().T @ M, y2)).real)

    assert abs(S_dense(q) - S0) < 1e-10 * S0
    F = ferm.force(q)
    eps = 1e-5
    for _ in range(8):
        mu, x = RNG.integers(4), RNG.integers(V)
        w = RNG.normal(size=3)
        fd = (S_dense(exp_update(q, mu, x, w, eps)) - S_dense(exp_update(q, mu, x, w, -eps))) / (2 * eps)
        assert abs(fd - F[mu, x] @ w) <= 1e-6 * max(1.0, abs(fd)), (fd, F[mu, x] @ w)


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.OMELYAN])
def test_hasenbusch_trajectory_reversible_and_second_order(integrator):
    dims = (4, 2, 2, 2)
    m0, m0_h, bc = 0.05, 0.5, 1
    q = smeared(dims, 71)
    p = momenta(dims, 72)
    eta, phi, _, _ = _hasenbusch_fields(dims, q, m0, m0_h, bc, 73)
    ferm = hmc.Hasenbusch(dims, m0, m0_h, eta, phi, bc=bc)
    q1, p1, i1 = hmc.trajectory(dims, q, p, 2.2, 4, 0.4, integrator, ferm)
    q2, p2, i2 = hmc.trajectory(dims, q1, -p1, 2.2, 4, 0.4, integrator, ferm)
    assert np.abs(q2 - q).max() < 1e-10 and np.abs(p2 + p).max() < 1e-9
    dh = [abs(hmc.trajectory(dims, q, p, 2.2, n, 0.5, integrator, ferm)[2]["dH"]) for n in (8, 16)]
    assert 3.8 < dh[0] / dh[1] < 4.2, dh


# ---------------------------------------------------------------- multiple time scales

class _NoFermions:
    """A pseudofermion term with zero action and zero force."""

    def action(self, q):
        return 0.0

    def force(self, q):
        return np.zeros((4, q.shape[1], 3))


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.OMELYAN])
def test_nested_inner_level_is_the_single_level_integrator(integrator):
    """With a vanishing outer force the two-level scheme is the gauge integrator
    alone: n outer steps of m inner steps are n m leapfrog steps, or 2 n m
    Omelyan steps (each outer Omelyan step drifts twice), of the single-level code."""
    dims = (4, 4, 2, 2)
    q = smeared(dims, 81)
    p = momenta(dims, 82)
    n, m = 3, 2
    q1, p1, _ = hmc.trajectory(dims, q, p, 2.2, n, 0.6, integrator, _NoFermions(), n_steps_gauge=m)
    k = n * m if integrator == hmc.LEAPFROG else 2 * n * m
    q2, p2, _ = hmc.trajectory(dims, q, p, 2.2, k, 0.6, integrator)
    assert np.abs(q1 - q2).max() < 1e-13 and np.abs(p1 - p2).max() < 1e-12


def test_nested_leapfrog_with_one_inner_step_is_leapfrog():
    """Momentum kicks commute, so one inner step per outer drift is plain leapfrog."""
    dims = (4, 2, 2, 2)
    m0 = 0.1
    q = smeared(dims, 83)
    p = momenta(dims, 84)
    ferm = hmc.Fermions(dims, m0, pseudofermion(dims, m0, 85), bc=1)
    q1, p1, i1 = hmc.trajectory(dims, q, p, 2.2, 3, 0.4, hmc.LEAPFROG, ferm)
    qn, pn = hmc.nested_steps(dims, q, p, 2.2, 3, 0.4 / 3, hmc.LEAPFROG, ferm, 1)
    assert np.abs(qn - q1).max() < 1e-12 and np.abs(pn - p1).max() < 1e-11


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.OMELYAN])
def test_nested_trajectory_reversible_and_second_order(integrator):
    dims = (4, 2, 2, 2)
    m0 = 0.1
    q = smeared(dims, 86)
    p = momenta(dims, 87)
    ferm = hmc.Fermions(dims, m0, pseudofermion(dims, m0, 88), bc=1)
    q1, p1, i1 = hmc.trajectory(dims, q, p, 2.2, 3, 0.4, integrator, ferm, n_steps_gauge=3)
    q2, p2, i2 = hmc.trajectory(dims, q1, -p1, 2.2, 3, 0.4, integrator, ferm, n_steps_gauge=3)
    assert np.abs(q2 - q).max() < 1e-10 and np.abs(p2 + p).max() < 1e-9
    assert abs(i1["dH"] + i2["dH"]) < 1e-9
    dh = [abs(hmc.trajectory(dims, q, p, 2.2, n, 0.5, integrator, ferm, n_steps_gauge=2)[2]["dH"])
          for n in (8, 16, 32)]
    assert 3.8 < dh[0] / dh[1] < 4.2 and 3.8 < dh[1] / dh[2] < 4.2, dh


def test_oracle_chain_creutz_equality():
    """<exp(-dH)> = 1 over an equilibrium chain of the oracle's own HMC (Wilson
    fermions, eta = Mhat^+ xi drawn with the oracle's Schur operator): the
    trajectory's area preservation and reversibility and the heat baths'
    normalisation together (deterministic seed; 4 standard errors)."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    beta, m0 = 2.0, 0.2
    rng = np.random.default_rng(91)
    q = smeared(dims, 92)
    even = oracle.parity_mask(dims) == 0
    w = []
    for it in range(240):
        p = rng.normal(size=(4, V, 3))
        xi = (rng.normal(size=(V, 4, 2)) + 1j * rng.normal(size=(V, 4, 2))) / np.sqrt(2.0)
        xi[~even] = 0
        eta = oracle.schur(dims, oracle.expand_links(dims, 2, q), m0, xi, dagger=True, bc=1)
        ferm = hmc.Fermions(dims, m0, eta, bc=1)
        q1, _, info = hmc.trajectory(dims, q, p, beta, 2, 1.0, hmc.OMELYAN, ferm)   # std(dH) about 0.2
        if it >= 40:
            w.append(np.exp(-info["dH"]))
        if rng.uniform() < np.exp(-info["dH"]):
            q = q1
    w = np.array(w)
    err = w.std(ddof=1) / np.sqrt(len(w))
    assert abs(w.mean() - 1.0) <= 4 * err + 1e-3, (w.mean(), err)
