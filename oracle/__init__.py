"""FP64 CPU oracle for the Wilson-Dirac operator (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It never touches the CUDA library and the CUDA
library never touches it.

Numpy wrappers around ``wilson_oracle.c`` (the plain-C definition of the
operator, its adjoint and a textbook CG on the normal equations), plus the
even-odd blocks written as restrictions of the same full-lattice loops:

* ``hop_block(p, in_half)``  = H_{p,1-p} in   (paper: Dslash restricted to one
  parity, section "Wilson inverter: Main features")
* ``schur(x_e)``             = (1 - kappa^2 H_eo H_oe) x_e   (paper Fig. 1's
  preconditioned operator)
* ``schur_rhs / schur_reconstruct`` = the standard Schur-complement algebra
  that turns D x = b into the even-site system and back.

Parity unpinned: none of these functions has a value printed in the paper
(the paper prints no worked example).  Every function is pinned by the
mathematics instead: free-field closed form, adjointness, gamma5-hermiticity,
gauge covariance, brute force on 2^4 and LAPACK solves.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        dp = C.c_void_p
        L.oracle_gamma.argtypes = [C.c_int, dp]
        L.oracle_hop.argtypes = [dp, dp, dp, dp, C.c_int, C.c_int]
        L.oracle_hop_sites.argtypes = [dp, dp, dp, dp, C.c_int, dp, C.c_long]
        L.oracle_apply_D.argtypes = [dp, dp, dp, dp, C.c_double, C.c_int]
        L.oracle_cgnr.argtypes = [dp, dp, dp, dp, C.c_double, C.c_double, C.c_int,
                                  C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.oracle_cgnr.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _vol(dims):
    d = [int(v) for v in dims]
    return d[0] * d[1] * d[2] * d[3]


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def gamma(mu: int) -> np.ndarray:
    """4x4 gamma matrix of the oracle's basis; mu = 4 gives gamma_5."""
    g = np.zeros(16, dtype=np.complex128)
    lib().oracle_gamma(int(mu), g.ctypes.data)
    return g.reshape(4, 4)


def hop(psi, U, dims, dagger: bool = False, out_parity: int = -1) -> np.ndarray:
    """H psi (or H^+ psi) on the full lattice; out_parity restricts the output."""
    psi = _c128(psi)
    U = _c128(U)
    d = _dims(dims)
    out = np.empty_like(psi)
    lib().oracle_hop(out.ctypes.data, psi.ctypes.data, U.ctypes.data, d.ctypes.data,
                     int(bool(dagger)), int(out_parity))
    return out


def hop_sites(psi, U, dims, sites, dagger: bool = False) -> np.ndarray:
    """H psi (or H^+ psi) at the given lexicographic sites: complex128[n, 4, 3]."""
    psi = _c128(psi)
    U = _c128(U)
    d = _dims(dims)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((len(s), 4, 3), dtype=np.complex128)
    lib().oracle_hop_sites(out.ctypes.data, psi.ctypes.data, U.ctypes.data, d.ctypes.data,
                           int(bool(dagger)), s.ctypes.data, len(s))
    return out


def apply_D(psi, U, dims, kappa: float, dagger: bool = False) -> np.ndarray:
    """D psi = psi - kappa H psi (dagger: D^+ psi = psi - kappa H^+ psi)."""
    psi = _c128(psi)
    U = _c128(U)
    d = _dims(dims)
    out = np.empty_like(psi)
    lib().oracle_apply_D(out.ctypes.data, psi.ctypes.data, U.ctypes.data, d.ctypes.data,
                         float(kappa), int(bool(dagger)))
    return out


def cgnr(b, U, dims, kappa: float, tol: float = 1e-10, maxiter: int = 10000, x0=None):
    """Solve D x = b with CG on D^+ D x = D^+ b.  Returns (x, iters, relres, ok)."""
    b = _c128(b)
    U = _c128(U)
    d = _dims(dims)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    it = C.c_int(0)
    rel = C.c_double(0)
    st = lib().oracle_cgnr(x.ctypes.data, b.ctypes.data, U.ctypes.data, d.ctypes.data,
                           float(kappa), float(tol), int(maxiter),
                           C.byref(it), C.byref(rel))
    return x, it.value, rel.value, st == 0


# ---------------------------------------------------------------------------
# even-odd blocks as restrictions of the full-lattice loops
# ---------------------------------------------------------------------------

def _parity(dims):
    L0, L1, L2, L3 = (int(v) for v in dims)
    i = np.arange(L0 * L1 * L2 * L3)
    x0 = i % L0
    x1 = (i // L0) % L1
    x2 = (i // (L0 * L1)) % L2
    x3 = i // (L0 * L1 * L2)
    return (x0 + x1 + x2 + x3) & 1


def embed(half, dims, parity: int) -> np.ndarray:
    """Half-lattice field of ``parity`` -> full lattice, zero on the other parity."""
    full = np.zeros((_vol(dims), 4, 3), dtype=np.complex128)
    full[_parity(dims) == parity] = half
    return full


def restrict(full, dims, parity: int) -> np.ndarray:
    return np.ascontiguousarray(full[_parity(dims) == parity])


def hop_block(out_parity: int, in_half, U, dims, dagger: bool = False) -> np.ndarray:
    """H_{p,1-p} in_half (or the block of H^+): half-lattice of parity p."""
    full = embed(in_half, dims, 1 - out_parity)
    return restrict(hop(full, U, dims, dagger, out_parity), dims, out_parity)


def schur(x_e, U, dims, kappa: float, dagger: bool = False) -> np.ndarray:
    """(1 - kappa^2 H_eo H_oe) x_e, or its adjoint with the H^+ blocks."""
    t = hop_block(1, x_e, U, dims, dagger)
    return np.asarray(x_e) - kappa * kappa * hop_block(0, t, U, dims, dagger)


def schur_rhs(b, U, dims, kappa: float) -> np.ndarray:
    """b_hat_e = b_e + kappa H_eo b_o."""
    return restrict(b, dims, 0) + kappa * hop_block(0, restrict(b, dims, 1), U, dims)


def schur_reconstruct(x_e, b, U, dims, kappa: float) -> np.ndarray:
    """x_o = b_o + kappa H_oe x_e, returned as the full-lattice solution."""
    x_o = restrict(b, dims, 1) + kappa * hop_block(1, x_e, U, dims)
    full = embed(x_e, dims, 0)
    full[_parity(dims) == 1] = x_o
    return full
