"""Seeded synthetic inputs for the Wilson-Dirac operator and its solves.

The paper benchmarks on unspecified gauge configurations; these generators
stand in for them with fields of the same structure.  Both the CPU oracle and
the CUDA path receive the arrays produced here and nothing else is shared.

Canonical (host, FP64) layouts
------------------------------
* site index (lexicographic): ``i = x0 + L0*(x1 + L1*(x2 + L2*x3))``, with
  ``x3`` the time direction.
* spinor field: ``complex128[V, 4, 3]`` (site, spin, colour).
* gauge field: ``complex128[4, V, 3, 3]`` (direction mu, site, row, column);
  ``U[mu, x]`` is the link from ``x`` to ``x + mu_hat``.
* half-lattice (one parity) arrays hold the sites of that parity in increasing
  lexicographic order, i.e. site ``i`` sits at position ``i >> 1``.

Recipes (seeds as documented in the design notes)
-------------------------------------------------
* links: ``U = reunit(exp(i * eps * H))``, ``H = (A + A^dagger)/2 - tr/3`` with
  ``A`` a 3x3 matrix of unit-variance complex normals; ``eps = 0.3``.
* spinors: complex normals with real and imaginary parts ~ N(0, 1/2).
* gauge transformations: the link recipe with ``eps = 1``.
"""
from __future__ import annotations

import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np

from . import rng

STREAM_LINKS = 1
STREAM_SPINOR = 2
STREAM_GAUGE_XFORM = 3

SEED_LINKS = 1234
SEED_SPINOR = 5678
SEED_OMEGA = 91011


def volume(dims) -> int:
    L0, L1, L2, L3 = (int(d) for d in dims)
    return L0 * L1 * L2 * L3


def coords(dims) -> np.ndarray:
    """int64[V, 4] coordinates of every lexicographic site index."""
    L0, L1, L2, L3 = (int(d) for d in dims)
    i = np.arange(volume(dims), dtype=np.int64)
    x0 = i % L0
    r = i // L0
    x1 = r % L1
    r //= L1
    x2 = r % L2
    x3 = r // L2
    return np.stack([x0, x1, x2, x3], axis=1)


def site_parity(dims) -> np.ndarray:
    return coords(dims).sum(axis=1) & 1


def half_sites(dims, parity: int) -> np.ndarray:
    """Lexicographic indices of the sites of ``parity``, increasing."""
    return np.nonzero(site_parity(dims) == parity)[0]


def to_half(full: np.ndarray, dims, parity: int) -> np.ndarray:
    return np.ascontiguousarray(full[half_sites(dims, parity)])


def from_halves(even: np.ndarray, odd: np.ndarray, dims) -> np.ndarray:
    full = np.zeros((volume(dims),) + even.shape[1:], dtype=even.dtype)
    full[half_sites(dims, 0)] = even
    full[half_sites(dims, 1)] = odd
    return full


# --------------------------------------------------------------------------
# SU(3) matrices
# --------------------------------------------------------------------------

def _hermitian_traceless(seed: int, stream: int, first: int, count: int) -> np.ndarray:
    a = rng.complex_normal(seed, stream, 9 * first, 9 * count).reshape(count, 3, 3)
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h[:, 0, 0] -= tr
    h[:, 1, 1] -= tr
    h[:, 2, 2] -= tr
    return h


def reunitarise(u: np.ndarray) -> np.ndarray:
    """Project onto SU(3): Gram-Schmidt the rows, then rotate row 2's phase
    so that the determinant is exactly 1 (up to rounding)."""
    u = np.array(u, dtype=np.complex128, copy=True)
    r0 = u[:, 0, :]
    r0 /= np.linalg.norm(r0, axis=1)[:, None]
    r1 = u[:, 1, :]
    r1 -= np.sum(np.conj(r0) * r1, axis=1)[:, None] * r0
    r1 /= np.linalg.norm(r1, axis=1)[:, None]
    r2 = u[:, 2, :]
    r2 -= np.sum(np.conj(r0) * r2, axis=1)[:, None] * r0
    r2 -= np.sum(np.conj(r1) * r2, axis=1)[:, None] * r1
    r2 /= np.linalg.norm(r2, axis=1)[:, None]
    det = np.linalg.det(u)
    r2 *= np.conj(det / np.abs(det))[:, None]
    return u


def _su3_chunk(args) -> np.ndarray:
    seed, stream, first, count, eps = args
    h = _hermitian_traceless(seed, stream, first, count)
    w, v = np.linalg.eigh(h)
    u = (v * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(v, 1, 2))
    return reunitarise(u)


def _su3_batch(seed: int, stream: int, count: int, eps: float,
               workers: int | None = None) -> np.ndarray:
    """``count`` SU(3) matrices; matrix j depends only on (seed, stream, j)."""
    chunk = 1 << 18
    jobs = [(seed, stream, s, min(chunk, count - s), eps) for s in range(0, count, chunk)]
    if workers is None:
        workers = min(len(jobs), os.cpu_count() or 1, 32)
    if workers <= 1 or len(jobs) <= 1:
        parts = [_su3_chunk(j) for j in jobs]
    else:
        # spawn: never fork a process that may already hold a CUDA context
        with ProcessPoolExecutor(max_workers=workers,
                                 mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_su3_chunk, jobs))
    return np.concatenate(parts, axis=0) if parts else np.zeros((0, 3, 3), np.complex128)


def su3_links(dims, seed: int = SEED_LINKS, eps: float = 0.3,
              workers: int | None = None) -> np.ndarray:
    """complex128[4, V, 3, 3]: U_mu(x) = reunit(exp(i eps H_mu(x)))."""
    V = volume(dims)
    return _su3_batch(seed, STREAM_LINKS, 4 * V, eps, workers).reshape(4, V, 3, 3)


def unit_links(dims) -> np.ndarray:
    V = volume(dims)
    u = np.zeros((4, V, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gauge_transform(dims, seed: int = SEED_OMEGA, eps: float = 1.0) -> np.ndarray:
    """complex128[V, 3, 3]: a random SU(3) matrix Omega(x) per site."""
    return _su3_batch(seed, STREAM_GAUGE_XFORM, volume(dims), eps, workers=1)


# --------------------------------------------------------------------------
# spinors
# --------------------------------------------------------------------------

def gaussian_spinor(dims, seed: int = SEED_SPINOR, nsites: int | None = None,
                    first_site: int = 0) -> np.ndarray:
    """complex128[V, 4, 3] with Re, Im ~ N(0, 1/2) per component."""
    V = volume(dims) if nsites is None else nsites
    z = rng.complex_normal(seed, STREAM_SPINOR, 12 * first_site, 12 * V, variance=1.0)
    return z.reshape(V, 4, 3)


def point_source(dims, site: int = 0, spin: int = 0, colour: int = 0) -> np.ndarray:
    psi = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    psi[site, spin, colour] = 1.0
    return psi
