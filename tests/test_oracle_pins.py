"""Pins for the FP64 oracle and the input generators (CPU only).

The paper prints no worked example, so every pin here comes from mathematics
the operator must satisfy, chosen so that a plausible slip in the oracle (a
projector sign, a dropped hop, a swapped link index, U where U^+ belongs, a
transposed link, a missing antiperiodic sign) fails at least one of them.
The last block plants such slips on the CPU and checks that the pins catch
them.
"""
import itertools

import numpy as np
import pytest

from synth import fields, rng

KAPPA = 0.12


def plane_wave(dims, n, chi):
    """e^{i p.x} chi with p_mu = 2 pi n_mu / L_mu (mu < 3) and the
    antiperiodic time momentum p_3 = (2 n_3 + 1) pi / L_3."""
    L = np.asarray(dims)
    p = np.array([2 * np.pi * n[0] / L[0], 2 * np.pi * n[1] / L[1],
                  2 * np.pi * n[2] / L[2], (2 * n[3] + 1) * np.pi / L[3]])
    x = fields.coords(dims)
    phase = np.exp(1j * (x @ p))
    return phase[:, None, None] * chi[None, :, :], p


def shift(field, dims, mu, step):
    """field(x + step * mu_hat), periodic, as a full-lattice array."""
    x = fields.coords(dims)
    y = x.copy()
    y[:, mu] = (y[:, mu] + step) % dims[mu]
    L0, L1, L2, _ = dims
    j = y[:, 0] + L0 * (y[:, 1] + L1 * (y[:, 2] + L2 * y[:, 3]))
    return field[j]


def gauge_rotate(U, omega, dims):
    """U'_mu(x) = Omega(x) U_mu(x) Omega(x + mu)^+."""
    out = np.empty_like(U)
    for mu in range(4):
        om_fwd = shift(omega, dims, mu, +1)
        out[mu] = omega @ U[mu] @ np.conj(np.swapaxes(om_fwd, 1, 2))
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# generator
# ---------------------------------------------------------------------------

def test_splitmix64_published_stream():
    # first outputs of sequential SplitMix64 seeded with 1234567, as published
    # with the reference implementation (Vigna, prng.di.unimi.it)
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    got = rng.raw_u64(1234567, 0, np.arange(5)).tolist()
    assert got == want


def test_normals_moments():
    z = rng.complex_normal(5678, 2, 0, 200000)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    assert abs(np.mean(z.real)) < 0.01 and abs(np.mean(z.imag)) < 0.01
    assert abs(np.var(z.real) - 0.5) < 0.01


def test_generator_chunk_independent():
    dims = (4, 4, 4, 4)
    a = fields.su3_links(dims, workers=1)
    b = fields._su3_batch(fields.SEED_LINKS, fields.STREAM_LINKS, 4 * 256, 0.3, workers=1)
    assert np.array_equal(a.reshape(-1, 3, 3), b)
    psi = fields.gaussian_spinor(dims)
    tail = fields.gaussian_spinor(dims, nsites=10, first_site=100)
    assert np.array_equal(psi[100:110], tail)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_links_are_su3(dims):
    U = fields.su3_links(dims).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.max(np.abs(np.conj(np.swapaxes(U, 1, 2)) @ U - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-14


def test_links_third_row_from_first_two():
    # the identity behind 12-real link compression (paper: "reading only two
    # columns of each gauge matrix and reconstructing the third"): for SU(3),
    # row 2 = conj(row 0 x row 1)
    U = fields.su3_links((4, 4, 4, 4)).reshape(-1, 3, 3)
    r2 = np.conj(np.cross(U[:, 0, :], U[:, 1, :]))
    assert np.max(np.abs(r2 - U[:, 2, :])) < 1e-14


def test_link_normalisation_mean():
    # eps = 0.3 with H = (A + A^+)/2 - tr/3: mean Re tr U / 3 close to 0.94
    U = fields.su3_links((4, 4, 4, 8)).reshape(-1, 3, 3)
    m = np.mean(np.trace(U, axis1=1, axis2=2).real) / 3
    assert 0.93 < m < 0.95


# ---------------------------------------------------------------------------
# gamma matrices
# ---------------------------------------------------------------------------

def test_gamma_clifford_and_hermitian(oracle):
    g = [oracle.gamma(m) for m in range(4)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            ac = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(ac, 2 * np.eye(4) * (a == b), atol=1e-15)


def test_gamma5_is_chiral(oracle):
    g5 = oracle.gamma(4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)
    assert np.allclose(g5, oracle.gamma(0) @ oracle.gamma(1) @ oracle.gamma(2) @ oracle.gamma(3))


# ---------------------------------------------------------------------------
# free field: closed form in momentum space
# ---------------------------------------------------------------------------

FREE_CASES = [
    ((4, 4, 4, 4), (0, 0, 0, 0)),
    ((4, 4, 4, 4), (1, 0, 2, 1)),
    ((4, 4, 4, 4), (3, 1, 1, 3)),
    ((4, 4, 4, 8), (1, 2, 3, 5)),
    ((4, 4, 4, 8), (0, 3, 1, 2)),
    ((2, 2, 2, 2), (1, 0, 1, 0)),
    ((6, 4, 2, 8), (5, 1, 1, 6)),
]


@pytest.mark.parametrize("dims,n", FREE_CASES)
def test_free_field_closed_form(oracle, dims, n):
    r = np.random.default_rng(7)
    chi = r.normal(size=(4, 3)) + 1j * r.normal(size=(4, 3))
    psi, p = plane_wave(dims, n, chi)
    U = fields.unit_links(dims)
    got = oracle.apply_D(psi, U, dims, KAPPA)
    # D psi = [1 - 2 kappa sum cos p + 2 i kappa sum gamma_mu sin p_mu] psi
    M = (1 - 2 * KAPPA * np.sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        M = M + 2j * KAPPA * np.sin(p[mu]) * oracle.gamma(mu)
    want = np.einsum("ab,xbc->xac", M, psi)
    assert rel(got, want) < 1e-14


@pytest.mark.parametrize("dims,n", FREE_CASES)
def test_free_field_norm_basis_free(oracle, dims, n):
    # |D psi|^2 = [(1 - 2k sum cos)^2 + 4k^2 sum sin^2] |psi|^2 for any
    # Hermitian Clifford basis: this does not use the oracle's gammas at all
    r = np.random.default_rng(11)
    chi = r.normal(size=(4, 3)) + 1j * r.normal(size=(4, 3))
    psi, p = plane_wave(dims, n, chi)
    out = oracle.apply_D(psi, fields.unit_links(dims), dims, KAPPA)
    lam = (1 - 2 * KAPPA * np.sum(np.cos(p))) ** 2 + 4 * KAPPA ** 2 * np.sum(np.sin(p) ** 2)
    assert abs(np.vdot(out, out).real / np.vdot(psi, psi).real - lam) < 1e-13


# ---------------------------------------------------------------------------
# adjoint, gamma5-hermiticity, gauge covariance
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 4)])
def test_adjoint_by_inner_products(oracle, dims):
    U = fields.su3_links(dims)
    x = fields.gaussian_spinor(dims, seed=1)
    y = fields.gaussian_spinor(dims, seed=2)
    lhs = np.vdot(y, oracle.apply_D(x, U, dims, KAPPA))
    rhs = np.vdot(oracle.apply_D(y, U, dims, KAPPA, dagger=True), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (4, 6, 2, 8)])
def test_gamma5_hermiticity(oracle, dims):
    U = fields.su3_links(dims)
    x = fields.gaussian_spinor(dims, seed=3)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    g5D = np.einsum("ab,xbc->xac", g5, oracle.apply_D(np.einsum("ab,xbc->xac", g5, x), U, dims, KAPPA))
    assert rel(oracle.apply_D(x, U, dims, KAPPA, dagger=True), g5D) < 1e-14


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (4, 2, 6, 4)])
def test_gauge_covariance(oracle, dims):
    U = fields.su3_links(dims)
    om = fields.gauge_transform(dims)
    x = fields.gaussian_spinor(dims, seed=4)
    Up = gauge_rotate(U, om, dims)
    lhs = oracle.apply_D(np.einsum("xab,xsb->xsa", om, x), Up, dims, KAPPA)
    rhs = np.einsum("xab,xsb->xsa", om, oracle.apply_D(x, U, dims, KAPPA))
    assert rel(lhs, rhs) < 1e-13


# ---------------------------------------------------------------------------
# brute force on 2^4 (each direction has 2 sites: x + mu = x - mu, both hops add)
# ---------------------------------------------------------------------------

def dense_wilson(U, dims, kappa, gam):
    """Dense 12V x 12V matrix of D by brute force over (site, site) pairs."""
    V = fields.volume(dims)
    X = fields.coords(dims)
    M = np.eye(12 * V, dtype=complex)
    for i, j in itertools.product(range(V), range(V)):
        for mu in range(4):
            d = (X[j, mu] - X[i, mu]) % dims[mu]
            other = all(X[j, n] == X[i, n] for n in range(4) if n != mu)
            if not other:
                continue
            if d == 1 % dims[mu]:      # j = i + mu
                sgn = -1.0 if (mu == 3 and X[i, 3] == dims[3] - 1) else 1.0
                blk = np.kron(np.eye(4) - gam[mu], U[mu, i])
                M[12 * i:12 * i + 12, 12 * j:12 * j + 12] -= kappa * sgn * blk
            if d == (dims[mu] - 1) % dims[mu]:   # j = i - mu
                sgn = -1.0 if (mu == 3 and X[i, 3] == 0) else 1.0
                blk = np.kron(np.eye(4) + gam[mu], U[mu, j].conj().T)
                M[12 * i:12 * i + 12, 12 * j:12 * j + 12] -= kappa * sgn * blk
    return M


def test_dense_brute_force_2x4(oracle):
    dims = (2, 2, 2, 2)
    U = fields.su3_links(dims)
    gam = [oracle.gamma(m) for m in range(4)]
    M = dense_wilson(U, dims, KAPPA, gam)
    x = fields.gaussian_spinor(dims, seed=9)
    got = oracle.apply_D(x, U, dims, KAPPA).reshape(-1)
    assert rel(got, M @ x.reshape(-1)) < 1e-14
    gotd = oracle.apply_D(x, U, dims, KAPPA, dagger=True).reshape(-1)
    assert rel(gotd, M.conj().T @ x.reshape(-1)) < 1e-14
    g5 = np.kron(np.eye(16), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.allclose(g5 @ M @ g5, M.conj().T, atol=1e-15)


def test_cgnr_against_lapack_2x4(oracle):
    dims = (2, 2, 2, 2)
    U = fields.su3_links(dims)
    gam = [oracle.gamma(m) for m in range(4)]
    M = dense_wilson(U, dims, 0.137, gam)
    b = fields.gaussian_spinor(dims, seed=10)
    x_lu = np.linalg.solve(M, b.reshape(-1))
    x, it, rr, ok = oracle.cgnr(b, U, dims, 0.137, tol=1e-12, maxiter=2000)
    assert ok and rr <= 1e-12
    assert rel(x.reshape(-1), x_lu) < 1e-9


def test_cgnr_true_residual_4x4(oracle):
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims)
    b = fields.gaussian_spinor(dims, seed=12)
    x, it, rr, ok = oracle.cgnr(b, U, dims, KAPPA, tol=1e-10, maxiter=2000)
    assert ok
    r = b - oracle.apply_D(x, U, dims, KAPPA)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


# ---------------------------------------------------------------------------
# even-odd structure
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 4)])
def test_hop_connects_opposite_parities(oracle, dims):
    U = fields.su3_links(dims)
    x = fields.gaussian_spinor(dims, seed=13)
    full = oracle.hop(x, U, dims)
    for p in (0, 1):
        blk = oracle.hop_block(p, oracle.restrict(x, dims, 1 - p), U, dims)
        assert rel(blk, oracle.restrict(full, dims, p)) < 1e-15
        blkd = oracle.hop_block(p, oracle.restrict(x, dims, 1 - p), U, dims, dagger=True)
        assert rel(blkd, oracle.restrict(oracle.hop(x, U, dims, dagger=True), dims, p)) < 1e-15


def test_schur_solve_reproduces_full_solve(oracle):
    dims = (4, 4, 2, 2)
    kappa = 0.137
    U = fields.su3_links(dims)
    b = fields.gaussian_spinor(dims, seed=14)
    Vh = fields.volume(dims) // 2
    # dense Schur operator by applying it to unit vectors
    cols = []
    for k in range(12 * Vh):
        e = np.zeros(12 * Vh, dtype=complex)
        e[k] = 1
        cols.append(oracle.schur(e.reshape(Vh, 4, 3), U, dims, kappa).reshape(-1))
    Mhat = np.stack(cols, axis=1)
    bh = oracle.schur_rhs(b, U, dims, kappa)
    xe = np.linalg.solve(Mhat, bh.reshape(-1)).reshape(Vh, 4, 3)
    x = oracle.schur_reconstruct(xe, b, U, dims, kappa)
    r = b - oracle.apply_D(x, U, dims, kappa)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-13
    # the adjoint Schur operator is the matrix adjoint
    y = fields.gaussian_spinor(dims, seed=15)[:Vh]
    lhs = oracle.schur(y, U, dims, kappa, dagger=True).reshape(-1)
    assert rel(lhs, Mhat.conj().T @ y.reshape(-1)) < 1e-13


def test_hop_sites_matches_full(oracle):
    dims = (4, 6, 2, 4)
    U = fields.su3_links(dims)
    x = fields.gaussian_spinor(dims, seed=16)
    sites = np.array([0, 5, 17, 95, 191])
    full = oracle.hop(x, U, dims, dagger=True)
    assert np.array_equal(oracle.hop_sites(x, U, dims, sites, dagger=True), full[sites])


def test_thread_count_does_not_change_results(oracle):
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims)
    x = fields.gaussian_spinor(dims)
    n = oracle.get_threads()
    oracle.set_threads(1)
    a = oracle.hop(x, U, dims)
    oracle.set_threads(max(2, n))
    b = oracle.hop(x, U, dims)
    oracle.set_threads(n)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# planted slips: each must be caught by one of the pins above
# ---------------------------------------------------------------------------

def test_pin_catches_projector_sign(oracle):
    # H^+ is H with the projector signs exchanged: it must fail the closed form
    dims, n = (4, 4, 4, 4), (1, 0, 2, 1)
    chi = np.ones((4, 3), dtype=complex)
    psi, p = plane_wave(dims, n, chi)
    got = oracle.apply_D(psi, fields.unit_links(dims), dims, KAPPA, dagger=True)
    M = (1 - 2 * KAPPA * np.sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        M = M + 2j * KAPPA * np.sin(p[mu]) * oracle.gamma(mu)
    want = np.einsum("ab,xbc->xac", M, psi)
    assert rel(got, want) > 1e-2


def test_pin_catches_periodic_time(oracle):
    # a periodic-in-time plane wave is not an eigenvector of the antiperiodic operator
    dims = (4, 4, 4, 4)
    x = fields.coords(dims)
    p = np.array([np.pi / 2, 0, np.pi, 2 * np.pi / 4])
    psi = np.exp(1j * (x @ p))[:, None, None] * np.ones((1, 4, 3))
    got = oracle.apply_D(psi, fields.unit_links(dims), dims, KAPPA)
    M = (1 - 2 * KAPPA * np.sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        M = M + 2j * KAPPA * np.sin(p[mu]) * oracle.gamma(mu)
    assert rel(got, np.einsum("ab,xbc->xac", M, psi)) > 1e-2


def test_pin_catches_transposed_links(oracle):
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims)
    om = fields.gauge_transform(dims)
    x = fields.gaussian_spinor(dims, seed=4)
    UT = np.swapaxes(U, 2, 3).copy()
    UTp = np.swapaxes(gauge_rotate(U, om, dims), 2, 3).copy()
    lhs = oracle.apply_D(np.einsum("xab,xsb->xsa", om, x), UTp, dims, KAPPA)
    rhs = np.einsum("xab,xsb->xsa", om, oracle.apply_D(x, UT, dims, KAPPA))
    assert rel(lhs, rhs) > 1e-2


def test_pin_catches_dagger_links(oracle):
    # U^+ in place of U on forward hops is the same as feeding U^+ links
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims)
    om = fields.gauge_transform(dims)
    x = fields.gaussian_spinor(dims, seed=5)
    Ud = np.conj(np.swapaxes(U, 2, 3)).copy()
    Udp = np.conj(np.swapaxes(gauge_rotate(U, om, dims), 2, 3)).copy()
    lhs = oracle.apply_D(np.einsum("xab,xsb->xsa", om, x), Udp, dims, KAPPA)
    rhs = np.einsum("xab,xsb->xsa", om, oracle.apply_D(x, Ud, dims, KAPPA))
    assert rel(lhs, rhs) > 1e-2
