"""Differentiation through the C ABI: DiracApply and EoSolve autograd
functions and the su(2) fermion force, against the oracle's analytic
derivatives and against central finite differences.

Finite-difference set-up (16^4 configuration): S = Re<eta, (Mhat^+ Mhat)^-1 eta>
with eta a Gaussian source restricted to the even sites of a 4^4 block, so that
S is O(100) and single-link derivatives near the block are O(1): with solves
to a relative residual of 1e-13 the finite-difference noise (1e-13 S / eps)
stays near 1e-6 of the derivatives, and the O(eps^2) truncation at
eps = 1e-5 is far below.  64 random directions per check, tolerance 1e-6
relative to the largest derivative checked.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2411_18511_gb300 import autograd as ag  # noqa: E402


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda")


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def test_dirac_apply_backward_matches_oracle(cuda):
    dims = (4, 6, 2, 6)
    m0 = 0.1
    q = synth.haar_links(dims, 201)
    psi = synth.gaussian_spinor(dims, 2, 202)
    g = synth.gaussian_spinor(dims, 2, 203)
    qt = torch.tensor(q, device=cuda, requires_grad=True)
    pt = torch.tensor(psi, device=cuda, requires_grad=True)
    y = ag.DiracApply.apply(qt, pt, dims, m0)
    L = oracle.expand_links(dims, 2, q)
    assert rel(y.detach().cpu().numpy(), oracle.dirac(dims, L, m0, psi)) <= 1e-13
    y.backward(torch.tensor(g, device=cuda))
    want_psi = oracle.gamma5(oracle.dirac(dims, L, m0, oracle.gamma5(g)))
    assert rel(pt.grad.cpu().numpy(), want_psi) <= 1e-13
    want_q = -0.5 * oracle.link_grad(dims, g, psi)
    assert rel(qt.grad.cpu().numpy(), want_q) <= 1e-13


def test_dirac_apply_gradient_is_torch_convention(cuda):
    """L = sum |D psi|^2: torch's grad is 2 D^+ D psi; check one FD direction in psi."""
    dims = (2, 4, 2, 4)
    q = torch.tensor(synth.haar_links(dims, 211), device=cuda)
    psi = torch.tensor(synth.gaussian_spinor(dims, 2, 212), device=cuda, requires_grad=True)
    loss = (ag.DiracApply.apply(q, psi, dims, 0.3).abs() ** 2).sum()
    loss.backward()
    d = torch.tensor(synth.gaussian_spinor(dims, 2, 213), device=cuda)
    eps = 1e-6
    with torch.no_grad():
        lp = (ag.DiracApply.apply(q, psi + eps * d, dims, 0.3).abs() ** 2).sum()
        lm = (ag.DiracApply.apply(q, psi - eps * d, dims, 0.3).abs() ** 2).sum()
    fd = (lp - lm).item() / (2 * eps)
    an = torch.sum((psi.grad.conj() * d).real).item()
    assert abs(fd - an) <= 1e-7 * abs(an)


def localized_source(dims, seed):
    eta = synth.gaussian_spinor(dims, 2, seed)
    x = np.indices(dims).reshape(4, -1).T
    inside = np.all(x < 4, axis=1) & (oracle.parity_mask(dims) == 0)
    eta[~inside] = 0
    return eta


@pytest.fixture(scope="module")
def field16():
    dims = (16, 16, 16, 16)
    q, _, _ = synth.ape_smear_to_plaquette(synth.haar_links(dims, 1005), dims, 0.6)
    return dims, q


def near_block_links(dims, rng, n):
    """Random (mu, site) pairs with the site within distance 2 of the source block."""
    x = np.indices(dims).reshape(4, -1).T
    near = np.where(np.all((x < 6) | (x >= np.array(dims) - 2), axis=1))[0]
    return rng.integers(0, 4, n), rng.choice(near, n)


def test_eo_solve_backward_vs_finite_differences(cuda, field16):
    dims, q = field16
    m0 = -0.2
    eta = localized_source(dims, 2005)
    qt = torch.tensor(q, device=cuda, requires_grad=True)
    et = torch.tensor(eta, device=cuda)
    x = ag.EoSolve.apply(qt, et, dims, m0, 1e-13)
    S = torch.sum(et.conj() * x).real
    S.backward()
    G = qt.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    mus, sites = near_block_links(dims, rng, 64)
    eps = 1e-5
    fds, ans = [], []
    with torch.no_grad():
        for mu, site in zip(mus, sites):
            d = rng.normal(size=4)
            d /= np.linalg.norm(d)
            vals = []
            for s in (+1, -1):
                qq = q.copy()
                qq[mu, site] += s * eps * d
                xx = ag.EoSolve.apply(torch.tensor(qq, device=cuda), et, dims, m0, 1e-13)
                vals.append(torch.sum(et.conj() * xx).real.item())
            fds.append((vals[0] - vals[1]) / (2 * eps))
            ans.append(G[mu, site] @ d)
    fds, ans = np.array(fds), np.array(ans)
    scale = np.abs(ans).max()
    assert scale > 1e-3
    assert np.max(np.abs(fds - ans)) <= 1e-6 * scale, np.max(np.abs(fds - ans)) / scale
    # grad_eta = A^-1 g with g = eta: equal to x itself for S = Re<eta, x>
    # (checked through the link gradient above; the source gradient below)


def su2_exp(w):
    th = np.linalg.norm(w) / 2
    return np.concatenate([[np.cos(th)], np.sin(th) * w / np.linalg.norm(w)])


def test_fermion_force_vs_finite_differences(cuda, field16):
    dims, q = field16
    m0 = -0.2
    eta = localized_source(dims, 2006)
    qt = torch.tensor(q, device=cuda)
    et = torch.tensor(eta, device=cuda)
    F, S0 = ag.fermion_force(qt, et, dims, m0, tol=1e-13)
    F = F.cpu().numpy()
    rng = np.random.default_rng(6)
    mus, sites = near_block_links(dims, rng, 64)
    eps = 1e-5
    diffs, ans = [], []
    for mu, site in zip(mus, sites):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        vals = []
        for s in (+1, -1):
            qq = q.copy()
            qq[mu, site] = synth.quat_mul(su2_exp(s * eps * w), q[mu, site])
            _, Sv = ag.fermion_force(torch.tensor(qq, device=cuda), et, dims, m0, tol=1e-13)
            vals.append(Sv.item())
        fd = (vals[0] - vals[1]) / (2 * eps)
        an = F[mu, site] @ w
        diffs.append(abs(fd - an))
        ans.append(abs(an))
    scale = max(ans)
    assert scale > 1e-3
    assert max(diffs) <= 1e-6 * scale, max(diffs) / scale


def test_force_and_eo_gradient_match_oracle_small(cuda):
    """GPU analytic derivatives equal the oracle's at 4^4 to 1e-12."""
    dims = (4, 4, 4, 4)
    m0 = 0.2
    q = synth.haar_links(dims, 221)
    eta = synth.gaussian_spinor(dims, 2, 222)
    eta[oracle.parity_mask(dims) == 1] = 0
    L = oracle.expand_links(dims, 2, q)
    X, it, tr, ok = oracle.cg(dims, L, m0, eta, tol=1e-14, maxiter=5000)
    Y = oracle.schur(dims, L, m0, X)
    even = oracle.parity_mask(dims) == 0
    Z = oracle.hop(dims, L, X, parity=1)
    W = oracle.gamma5(oracle.hop(dims, L, oracle.gamma5(Y), parity=1))
    a = np.where(even[:, None, None], Y, W)
    b = np.where(even[:, None, None], X, Z)
    c = 1.0 / (4 * (4 + m0))
    F_or = 2 * c * oracle.force(dims, L, a, b)
    F, _ = ag.fermion_force(torch.tensor(q, device=cuda), torch.tensor(eta, device=cuda), dims, m0, tol=1e-13)
    assert rel(F.cpu().numpy(), F_or) <= 1e-10
    # quaternion gradient of S = Re<eta, A^-1 eta> is 2c * link_grad((Y, W), (X, Z))
    qt = torch.tensor(q, device=cuda, requires_grad=True)
    x = ag.EoSolve.apply(qt, torch.tensor(eta, device=cuda), dims, m0, 1e-13)
    torch.sum(torch.tensor(eta, device=cuda).conj() * x).real.backward()
    G_or = 2 * c * oracle.link_grad(dims, a, b)
    assert rel(qt.grad.cpu().numpy(), G_or) <= 1e-10
