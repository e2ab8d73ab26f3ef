"""Plain FP64 CPU oracle for the even-odd Wilson-Dirac path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_2411_18511_gb300``; neither imports the other.  The arithmetic lives
in ``hr_oracle.c`` (plain C99, FP64, straight from the operator's definition);
this module only compiles it with gcc and marshals numpy arrays through ctypes.

Operator readings (the paper, arXiv:2411.18511, names the unimproved
Wilson-Dirac operator in Sec. 2.1 / Table 1 and its even-odd preconditioned
form in Sec. 2.1 without writing either down):

* ``D = (4+m0) - H/2`` with
  ``(H psi)(x) = sum_mu (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu)``,
  chiral gamma basis, periodic in every direction except those whose bit is set
  in ``bc`` (bit mu: antiperiodic, ``psi(x + L_mu mu) = -psi(x)``) or whose
  twist angle ``theta[mu]`` is nonzero (``psi(x + L_mu mu) = e^{i theta_mu}
  psi(x)``; with the bit as well, the product of both factors).  ``bc`` and
  ``theta`` are keywords of every operator below; a ``dims`` object with ``bc``
  and ``theta`` attributes supplies them too.
* ``Mhat = (4+m0) - H_eo H_oe / (4 (4+m0))`` on even sites, ``Mhat^+ = g5 Mhat g5``.
* CG: Hestenes-Stiefel on ``Mhat^+ Mhat`` from ``x0 = 0``.

Every function is pinned by tests/test_oracle_*.py against closed forms
(free field, flat connection), invariants (gamma5-hermiticity, gauge
covariance), an independent dense-matrix build, and finite differences.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hr_oracle.c with gcc (OpenMP over sites) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_long
            D = ctypes.c_double
            sig = {
                "or_expand_links": [P, I, P, P],
                "or_hop": [P, I, P, I, P, I, P, P],
                "or_hop_sites": [P, I, P, I, P, P, L, P, P],
                "or_dirac": [P, I, P, I, P, D, P, P],
                "or_schur": [P, I, P, I, P, D, I, P, P],
                "or_normal": [P, I, P, I, P, D, P, P],
                "or_cg": [P, I, P, I, P, D, P, P, D, I, P, P],
                "or_force": [P, I, P, P, P, P, P],
                "or_link_grad": [P, I, P, P, P, P],
                "or_plaquette": [P, P, P],
                "or_gamma": [I, P],
                "or_adjoint_link": [P, P],
                "or_num_threads": [],
                "or_set_num_threads": [I],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = I
            _lib = lib
    return _lib


def _dims(dims) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    assert d.shape == (4,)
    return d


def _bc(dims, bc) -> int:
    """Boundary bits: the explicit keyword, else the ``bc`` attribute of ``dims``, else 0."""
    b = int(bc) if bc is not None else int(getattr(dims, "bc", 0))
    if not 0 <= b <= 15:
        raise ValueError(f"bc = {b}: four bits, one per direction")
    return b


def _theta(dims, theta):
    """Twist angles: the explicit keyword, else the ``theta`` attribute of ``dims``;
    a float64[4] array kept alive by the caller, or None (no twist)."""
    t = theta if theta is not None else getattr(dims, "theta", None)
    if t is None:
        return None
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    if t.shape != (4,) or not np.all(np.isfinite(t)):
        raise ValueError("theta: four finite angles, one per direction")
    return t if np.any(t != 0.0) else None


def _tp(t):
    return None if t is None else t.ctypes.data_as(ctypes.c_void_p)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc: int, name: str):
    if rc < 0:
        raise ValueError(f"oracle {name} failed with code {rc}")


def volume(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> int:
    """Threads of the oracle's parallel loops from now on; returns the previous count."""
    return int(_load().or_set_num_threads(int(n)))


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3) or gamma5 (mu = 4) as a 4x4 complex matrix."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _check(_load().or_gamma(int(mu), _ptr(out)), "gamma")
    return out


def adjoint_link(q) -> np.ndarray:
    """R_ab = 1/2 tr(s_a U s_b U^+) for one quaternion q."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros((3, 3))
    _load().or_adjoint_link(_ptr(q), _ptr(R))
    return R


def expand_links(dims, nc: int, q) -> np.ndarray:
    """Colour matrices [4, V, nc, nc] (complex) from quaternion links [4, V, 4]."""
    d = _dims(dims)
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.shape == (4, volume(dims), 4)
    L = np.zeros((4, volume(dims), nc, nc), dtype=np.complex128)
    _check(_load().or_expand_links(_ptr(d), int(nc), _ptr(q), _ptr(L)), "expand_links")
    return L


def _nc(L) -> int:
    return int(L.shape[-1])


def hop(dims, L, psi, parity: int = -1, out=None, bc=None, theta=None) -> np.ndarray:
    """(H psi)(x) at the sites of ``parity`` (-1 = all); others stay zero (or as in ``out``)."""
    d = _dims(dims)
    th = _theta(dims, theta)
    psi = _c128(psi)
    out = np.zeros_like(psi) if out is None else out
    _check(_load().or_hop(_ptr(d), _bc(dims, bc), _tp(th), _nc(L), _ptr(L), int(parity), _ptr(psi), _ptr(out)),
           "hop")
    return out


def hop_sites(dims, L, psi, sites, bc=None, theta=None) -> np.ndarray:
    """(H psi) at the listed lexicographic sites, shape [n, 4, nc]."""
    d = _dims(dims)
    th = _theta(dims, theta)
    psi = _c128(psi)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((s.size, 4, _nc(L)), dtype=np.complex128)
    _check(_load().or_hop_sites(_ptr(d), _bc(dims, bc), _tp(th), _nc(L), _ptr(L), _ptr(s), s.size, _ptr(psi),
                                _ptr(out)),
           "hop_sites")
    return out


def dirac(dims, L, m0: float, psi, bc=None, theta=None) -> np.ndarray:
    """Full Wilson-Dirac operator D psi on all sites."""
    d = _dims(dims)
    th = _theta(dims, theta)
    psi = _c128(psi)
    out = np.zeros_like(psi)
    _check(_load().or_dirac(_ptr(d), _bc(dims, bc), _tp(th), _nc(L), _ptr(L), float(m0), _ptr(psi), _ptr(out)),
           "dirac")
    return out


def schur(dims, L, m0: float, psi, dagger: bool = False, bc=None, theta=None) -> np.ndarray:
    """Mhat psi (or Mhat^+ psi) on even sites of a full-lattice array; odd sites -> 0."""
    d = _dims(dims)
    th = _theta(dims, theta)
    psi = _c128(psi)
    out = np.zeros_like(psi)
    _check(_load().or_schur(_ptr(d), _bc(dims, bc), _tp(th), _nc(L), _ptr(L), float(m0), int(bool(dagger)), _ptr(psi),
                            _ptr(out)), "schur")
    return out


def normal(dims, L, m0: float, psi, bc=None, theta=None) -> np.ndarray:
    """Mhat^+ Mhat psi on even sites."""
    d = _dims(dims)
    th = _theta(dims, theta)
    psi = _c128(psi)
    out = np.zeros_like(psi)
    _check(_load().or_normal(_ptr(d), _bc(dims, bc), _tp(th), _nc(L), _ptr(L), float(m0), _ptr(psi), _ptr(out)),
           "normal")
    return out


def cg(dims, L, m0: float, b, tol: float = 1e-10, maxiter: int = 10000, bc=None, theta=None):
    """CG on Mhat^+ Mhat x = b (even sites). Returns (x, iters, true_rel_residual, converged)."""
    d = _dims(dims)
    th = _theta(dims, theta)
    b = _c128(b)
    x = np.zeros_like(b)
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    rc = _load().or_cg(_ptr(d), _bc(dims, bc), _tp(th), _nc(L), _ptr(L), float(m0), _ptr(b), _ptr(x), float(tol),
                       int(maxiter), ctypes.byref(it), ctypes.byref(tr))
    _check(rc, "cg")
    return x, it.value, tr.value, rc == 0


def force(dims, L, a, b, bc=None, theta=None) -> np.ndarray:
    """F[mu, x, a] = d Re<a, H b> / d w_a under U_mu(x) -> exp(i w.s/2) U_mu(x) (fundamental)."""
    d = _dims(dims)
    th = _theta(dims, theta)
    assert _nc(L) == 2
    a, b = _c128(a), _c128(b)
    F = np.zeros((4, volume(dims), 3))
    _check(_load().or_force(_ptr(d), _bc(dims, bc), _tp(th), _ptr(L), _ptr(a), _ptr(b), _ptr(F)), "force")
    return F


def link_grad(dims, a, b, bc=None, theta=None) -> np.ndarray:
    """G[mu, x, k] = d Re<a, H b> / d q_k for the quaternion components of U_mu(x)."""
    d = _dims(dims)
    th = _theta(dims, theta)
    a, b = _c128(a), _c128(b)
    G = np.zeros((4, volume(dims), 4))
    _check(_load().or_link_grad(_ptr(d), _bc(dims, bc), _tp(th), _ptr(a), _ptr(b), _ptr(G)), "link_grad")
    return G


def plaquette(dims, q) -> float:
    d = _dims(dims)
    q = np.ascontiguousarray(q, dtype=np.float64)
    P = ctypes.c_double(0.0)
    _check(_load().or_plaquette(_ptr(d), _ptr(q), ctypes.byref(P)), "plaquette")
    return P.value


# ---------------------------------------------------------------------------
# Composite steps built from the functions above (even-odd solve of D x = b)
# ---------------------------------------------------------------------------

def parity_mask(dims) -> np.ndarray:
    t, l1, l2, l3 = dims
    x = np.indices((t, l1, l2, l3)).sum(axis=0) & 1
    return x.reshape(-1)


def gamma5(psi) -> np.ndarray:
    g5 = np.diag(gamma(4))
    return psi * g5[None, :, None]


def eo_source(dims, L, m0: float, b, bc=None, theta=None) -> np.ndarray:
    """bhat_e = b_e - D_eo D_oo^-1 b_o = b_e + H_eo b_o / (2 (4+m0)); odd sites zero."""
    odd = parity_mask(dims) == 1
    bo = _c128(b).copy()
    bo[~odd] = 0
    h = hop(dims, L, bo, parity=0, bc=bc, theta=theta)
    out = _c128(b) + h / (2.0 * (4.0 + m0))
    out[odd] = 0
    return out


def eo_reconstruct(dims, L, m0: float, b, xe, bc=None, theta=None) -> np.ndarray:
    """x_o = D_oo^-1 (b_o - D_oe x_e) = (b_o + H_oe x_e / 2) / (4+m0); returns full x."""
    odd = parity_mask(dims) == 1
    h = hop(dims, L, _c128(xe), parity=1, bc=bc, theta=theta)
    x = _c128(xe).copy()
    x[odd] = (_c128(b)[odd] + 0.5 * h[odd]) / (4.0 + m0)
    return x
