"""Independent dense-matrix construction of the Wilson-Dirac operator (test pin).

Written separately from the oracle (no shared code): the gamma matrices are
spelled out entry by entry, links come from the explicit 2x2 form of a
quaternion and the adjoint links from the quaternion rotation matrix, and the
operator is assembled as a (4 nc V)^2 matrix from permutation matrices.  Used
on lattices up to 4^4 to brute-force the oracle's matrix-free routines.
"""

from __future__ import annotations

import numpy as np

# Chiral basis, written out: g0 = [[0,1],[1,0]], gk = [[0,-i s_k],[i s_k,0]].
_i = 1j
GAMMA = [
    np.array([[0, 0, 1, 0],
              [0, 0, 0, 1],
              [1, 0, 0, 0],
              [0, 1, 0, 0]], dtype=complex),
    np.array([[0, 0, 0, -_i],
              [0, 0, -_i, 0],
              [0, _i, 0, 0],
              [_i, 0, 0, 0]], dtype=complex),
    np.array([[0, 0, 0, -1],
              [0, 0, 1, 0],
              [0, 1, 0, 0],
              [-1, 0, 0, 0]], dtype=complex),
    np.array([[0, 0, -_i, 0],
              [0, 0, 0, _i],
              [_i, 0, 0, 0],
              [0, -_i, 0, 0]], dtype=complex),
]
GAMMA5 = np.diag([-1, -1, 1, 1]).astype(complex)


def su2(q) -> np.ndarray:
    """Explicit 2x2 matrix of a0 + i(a1 s1 + a2 s2 + a3 s3)."""
    a0, a1, a2, a3 = q
    return np.array([[a0 + 1j * a3, a2 + 1j * a1],
                     [-a2 + 1j * a1, a0 - 1j * a3]])


def rotation(q) -> np.ndarray:
    """Adjoint link as the 3x3 rotation of the unit quaternion q:
    R = (a0^2 - |a|^2) 1 + 2 a a^T + 2 a0 [a]_x^T, where [a]_x^T has entries eps_{b c k} a_k.
    """
    a0 = q[0]
    a = np.asarray(q[1:], dtype=float)
    cross = np.array([[0.0, a[2], -a[1]],
                      [-a[2], 0.0, a[0]],
                      [a[1], -a[0], 0.0]])
    return (a0 * a0 - a @ a) * np.eye(3) + 2.0 * np.outer(a, a) + 2.0 * a0 * cross


def site_index(dims):
    return np.arange(int(np.prod(dims))).reshape(dims)


def link_matrices(dims, q, nc):
    V = int(np.prod(dims))
    out = np.zeros((4, V, nc, nc), dtype=complex)
    for mu in range(4):
        for x in range(V):
            out[mu, x] = su2(q[mu, x]) if nc == 2 else rotation(q[mu, x])
    return out


def hopping_dense(dims, q, nc, bc=0, theta=None) -> np.ndarray:
    """Dense H with (H psi)(x) = sum_mu (1-g) U_mu(x) psi(x+mu) + (1+g) U_mu(x-mu)^+ psi(x-mu).

    Index order (site, spin, colour).  On an extent-2 direction the forward and
    backward neighbours coincide and the two blocks add.  Bit mu of ``bc`` makes
    direction mu antiperiodic: a block whose neighbour is reached through the
    lattice's edge in that direction enters with a minus sign.  A twist angle
    ``theta[mu]`` multiplies such a block by e^{+i theta_mu} when the neighbour
    is reached forward, e^{-i theta_mu} when backward.
    """
    V = int(np.prod(dims))
    idx = site_index(dims)
    xs = np.indices(dims).reshape(4, -1)  # xs[mu, x] = coordinate mu of site x
    U = link_matrices(dims, q, nc)
    n = V * 4 * nc
    H = np.zeros((V, 4, nc, V, 4, nc), dtype=complex)
    one = np.eye(4)
    for mu in range(4):
        fwd = np.roll(idx, -1, axis=mu).reshape(-1)  # fwd[x] = x + mu
        bwd = np.roll(idx, 1, axis=mu).reshape(-1)   # bwd[x] = x - mu
        anti = (bc >> mu) & 1
        tw = 0.0 if theta is None else float(theta[mu])
        pm = one - GAMMA[mu]
        pp = one + GAMMA[mu]
        for x in range(V):
            sf = sb = 1.0 + 0j
            if xs[mu, x] == dims[mu] - 1:
                sf = (-1.0 if anti else 1.0) * np.exp(1j * tw)
            if xs[mu, x] == 0:
                sb = (-1.0 if anti else 1.0) * np.exp(-1j * tw)
            H[x, :, :, fwd[x], :, :] += sf * np.einsum("st,cd->sctd", pm, U[mu, x])
            H[x, :, :, bwd[x], :, :] += sb * np.einsum("st,cd->sctd", pp, U[mu, bwd[x]].conj().T)
    return H.reshape(n, n)


def dirac_dense(dims, q, nc, m0, bc=0, theta=None) -> np.ndarray:
    n = int(np.prod(dims)) * 4 * nc
    return (4.0 + m0) * np.eye(n) - 0.5 * hopping_dense(dims, q, nc, bc, theta)


def parity_of_sites(dims) -> np.ndarray:
    return (np.indices(dims).sum(axis=0) & 1).reshape(-1)


def eo_blocks(dims, nc, M):
    """Split a (site, spin, colour) matrix into even/odd blocks."""
    par = np.repeat(parity_of_sites(dims), 4 * nc)
    e = np.where(par == 0)[0]
    o = np.where(par == 1)[0]
    return M[np.ix_(e, e)], M[np.ix_(e, o)], M[np.ix_(o, e)], M[np.ix_(o, o)], e, o


# ---------------------------------------------------------------- clover term

def sigma_dense(mu, nu) -> np.ndarray:
    """s_mn = (i/2)(g_mu g_nu - g_nu g_mu)."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


def clover_site_dense(dims, q, nc, m0, csw, exponential=False) -> np.ndarray:
    """Site matrices A(x) [V, 4 nc, 4 nc], site by site with explicit loops:
    the four leaves of each plane walked link by link from the explicit link
    matrices, F = (Q - Q^+)/8, C = (i/4) sum_{mu != nu} s_mn (x) F_mn,
    A = (4+m0) + csw C, or (4+m0) expm(csw C / (4+m0))."""
    from scipy.linalg import expm

    V = int(np.prod(dims))
    U = link_matrices(dims, q, nc)
    xs = np.indices(dims).reshape(4, -1).T
    idx = site_index(dims)

    def at(x):
        return idx[tuple(np.mod(x, dims))]

    def step(x, mu, s):
        y = np.array(x)
        y[mu] += s
        return y

    def link(x, mu, s):
        """the matrix that transports along one step: +1 U_mu(x), -1 U_mu(x - mu)^+"""
        if s > 0:
            return U[mu, at(x)]
        return U[mu, at(step(x, mu, -1))].conj().T

    def loop(x, path):
        m = np.eye(nc, dtype=complex)
        y = np.array(x)
        for mu, s in path:
            m = m @ link(y, mu, s)
            y = step(y, mu, s)
        assert np.all(np.mod(y, dims) == np.mod(x, dims))
        return m

    A = np.zeros((V, 4 * nc, 4 * nc), dtype=complex)
    a = 4.0 + m0
    for k in range(V):
        x = xs[k]
        C = np.zeros((4 * nc, 4 * nc), dtype=complex)
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                Q = (loop(x, [(mu, 1), (nu, 1), (mu, -1), (nu, -1)])
                     + loop(x, [(nu, 1), (mu, -1), (nu, -1), (mu, 1)])
                     + loop(x, [(mu, -1), (nu, -1), (mu, 1), (nu, 1)])
                     + loop(x, [(nu, -1), (mu, 1), (nu, 1), (mu, -1)]))
                F = (Q - Q.conj().T) / 8.0
                C += 0.25j * np.kron(sigma_dense(mu, nu), F)
        A[k] = expm(csw * C / a) * a if exponential else a * np.eye(4 * nc) + csw * C
    return A


def dirac_clover_dense(dims, q, nc, A, bc=0, theta=None) -> np.ndarray:
    """Dense D = A - H/2 with the site matrices A on the diagonal blocks."""
    V = int(np.prod(dims))
    n = V * 4 * nc
    D = -0.5 * hopping_dense(dims, q, nc, bc, theta)
    for x in range(V):
        s = slice(x * 4 * nc, (x + 1) * 4 * nc)
        D[s, s] += A[x]
    return D
