"""Seeded synthetic field generators.

Conventions shared with every consumer of these arrays:

* Lattice extents ``dims = (T, L1, L2, L3)``; the site ``x = (x0, x1, x2, x3)``
  (``x0`` is time) has lexicographic index
  ``i = ((x0*L1 + x1)*L2 + x2)*L3 + x3`` (``x3`` fastest).
* Gauge field: ``float64`` array of shape ``(4, V, 4)``: direction mu, site,
  quaternion ``(a0, a1, a2, a3)`` with ``a0^2+|a|^2 = 1``.  The SU(2) link it
  stands for is ``U = a0*1 + i*(a1*s1 + a2*s2 + a3*s3)`` (Pauli matrices s_k).
* Spinor field: ``complex128`` array of shape ``(V, 4, nc)``: site, spin,
  colour (``nc = 2`` fundamental, ``nc = 3`` adjoint).

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a
counter-based generator, through numpy's ``Generator(Philox(key=seed))``.
Normal deviates are drawn with the Box-Muller transform from its uniform
doubles, so the stream depends only on the published Philox definition and
not on numpy's normal sampler.
"""

from __future__ import annotations

import numpy as np


def lattice_volume(dims) -> int:
    t, l1, l2, l3 = (int(d) for d in dims)
    return t * l1 * l2 * l3


class Rng:
    """Philox4x32-10 stream keyed by ``seed``, with Box-Muller normals."""

    def __init__(self, seed: int):
        self._gen = np.random.Generator(np.random.Philox(key=int(seed)))

    def uniform(self, n: int) -> np.ndarray:
        return self._gen.random(int(n))

    def normal(self, n: int) -> np.ndarray:
        n = int(n)
        m = (n + 1) // 2
        u1 = 1.0 - self._gen.random(m)  # (0, 1]
        u2 = self._gen.random(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return z[:n]


def haar_quaternions(n: int, rng: Rng) -> np.ndarray:
    """``n`` Haar-distributed SU(2) elements as unit quaternions, shape (n, 4).

    A 4-vector of independent standard normals divided by its length is
    uniform on the 3-sphere, which is Haar measure on SU(2).
    """
    g = rng.normal(4 * n).reshape(n, 4)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def haar_links(dims, seed: int) -> np.ndarray:
    """Haar-random gauge field, shape (4, V, 4)."""
    v = lattice_volume(dims)
    return haar_quaternions(4 * v, Rng(seed)).reshape(4, v, 4)


def identity_links(dims) -> np.ndarray:
    v = lattice_volume(dims)
    q = np.zeros((4, v, 4))
    q[..., 0] = 1.0
    return q


def gaussian_spinor(dims, nc: int, seed: int, n_rhs: int | None = None) -> np.ndarray:
    """Gaussian complex source: every real and imaginary part ~ N(0, 1).

    Shape (V, 4, nc), or (n_rhs, V, 4, nc) when ``n_rhs`` is given.
    """
    v = lattice_volume(dims)
    k = 1 if n_rhs is None else int(n_rhs)
    z = Rng(seed).normal(2 * k * v * 4 * nc).reshape(k, v, 4, nc, 2)
    psi = z[..., 0] + 1j * z[..., 1]
    return psi[0] if n_rhs is None else psi


# ---------------------------------------------------------------------------
# Quaternion algebra used to synthesise smooth gauge fields (input preparation)
# ---------------------------------------------------------------------------

def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Product of the SU(2) elements a and b, in quaternion components.

    (a0 + i a.s)(b0 + i b.s) = (a0 b0 - a.b) + i (a0 b + b0 a - a x b).s
    """
    a0, av = a[..., 0], a[..., 1:]
    b0, bv = b[..., 0], b[..., 1:]
    out = np.empty(np.broadcast(a, b).shape)
    out[..., 0] = a0 * b0 - np.sum(av * bv, axis=-1)
    out[..., 1:] = a0[..., None] * bv + b0[..., None] * av - np.cross(av, bv)
    return out


def quat_conj(a: np.ndarray) -> np.ndarray:
    out = a.copy()
    out[..., 1:] *= -1.0
    return out


def _soa(q: np.ndarray, dims) -> np.ndarray:
    """(4, V, 4) links -> (4 mu, 4 comp, T, L1, L2, L3), components contiguous."""
    t, l1, l2, l3 = dims
    return np.ascontiguousarray(np.moveaxis(q.reshape(4, t, l1, l2, l3, 4), -1, 1))


def _aos(u: np.ndarray, dims) -> np.ndarray:
    return np.ascontiguousarray(np.moveaxis(u, 1, -1)).reshape(4, lattice_volume(dims), 4)


def _qmul(a, b, conj_a=False, conj_b=False):
    """Quaternion (SU(2)) product on component-major arrays (4, ...)."""
    a0, a1, a2, a3 = a[0], a[1], a[2], a[3]
    b0, b1, b2, b3 = b[0], b[1], b[2], b[3]
    if conj_a:
        a1, a2, a3 = -a1, -a2, -a3
    if conj_b:
        b1, b2, b3 = -b1, -b2, -b3
    out = np.empty(np.broadcast_shapes(a.shape, b.shape))
    out[0] = a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3
    out[1] = a0 * b1 + b0 * a1 - (a2 * b3 - a3 * b2)
    out[2] = a0 * b2 + b0 * a2 - (a3 * b1 - a1 * b3)
    out[3] = a0 * b3 + b0 * a3 - (a1 * b2 - a2 * b1)
    return out


def _shift(x, axis, step):
    """x(y + step * axis-hat) for component-major fields (lattice axes start at 1)."""
    return np.roll(x, -step, axis=axis + 1)


def _plaquette_soa(u) -> float:
    acc = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            p = _qmul(u[mu], _shift(u[nu], mu, 1))
            p = _qmul(p, _shift(u[mu], nu, 1), conj_b=True)
            acc += float(np.sum(_qmul(p, u[nu], conj_b=True)[0]))
    return acc / (6.0 * u[0, 0].size)


def mean_plaquette(q: np.ndarray, dims) -> float:
    """<P> = (1/6V) sum_{x, mu<nu} (1/2) Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+.

    For a quaternion, (1/2) Re tr U = a0.
    """
    return _plaquette_soa(_soa(q, dims))


def _staples(u):
    """Sum over nu != mu of the forward and backward staples of every link."""
    st = np.zeros_like(u)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            # forward: U_nu(x) U_mu(x+nu) U_nu(x+mu)^+
            s = _qmul(u[nu], _shift(u[mu], nu, 1))
            st[mu] += _qmul(s, _shift(u[nu], mu, 1), conj_b=True)
            # backward: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu)
            unm = _shift(u[nu], nu, -1)
            s = _qmul(unm, _shift(u[mu], nu, -1), conj_a=True)
            st[mu] += _qmul(s, _shift(unm, mu, 1))
    return st


def _ape_mix(u, st, alpha):
    # a real combination of SU(2) elements is a real multiple of one:
    # projecting back onto SU(2) is normalising the quaternion
    w = (1.0 - alpha) * u + (alpha / 6.0) * st
    return w / np.sqrt(np.sum(w * w, axis=1, keepdims=True))


def ape_smear_to_plaquette(q: np.ndarray, dims, target: float = 0.6,
                           alpha: float = 0.5, max_steps: int = 50):
    """APE-smear ``q`` until the mean plaquette reaches ``target``.

    The last step's weight is bisected so that the final plaquette lands
    within 1e-3 of ``target`` instead of overshooting it.  Returns
    ``(q_smeared, n_steps, plaquette)``.
    """
    u = _soa(q, dims)
    p = _plaquette_soa(u)
    steps = 0
    while p < target and steps < max_steps:
        st = _staples(u)
        nxt = _ape_mix(u, st, alpha)
        pn = _plaquette_soa(nxt)
        steps += 1
        if pn <= target + 1e-3:
            u, p = nxt, pn
            continue
        lo, hi = 0.0, alpha
        trial, pt = nxt, pn
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            trial = _ape_mix(u, st, mid)
            pt = _plaquette_soa(trial)
            if abs(pt - target) < 1e-3:
                break
            if pt < target:
                lo = mid
            else:
                hi = mid
        u, p = trial, pt
        break
    return _aos(u, dims), steps, p
