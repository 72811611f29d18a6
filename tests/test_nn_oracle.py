"""Pins of the network oracle (CPU): the numpy layer definition against the C
oracle's hopping term, gauge covariance, and the adjoint rule that the GPU
backward pass uses."""
import numpy as np
import pytest

import oracle
from oracle import nn
from synth import fields
from tests.test_oracle_pins import gauge_rotate


def hopping_weights(kappa, c, cin, cout):
    """(1 + c kappa H) on channels 0..3, identity on the remaining channels,
    from the C oracle's gamma matrices."""
    W = np.zeros((9, cout, cin), dtype=complex)
    for o in range(min(cin, cout)):
        W[0, o, o] = 1.0
    for mu in range(4):
        g = oracle.gamma(mu)
        W[1 + 2 * mu, :4, :4] = c * kappa * (np.eye(4) - g)
        W[2 + 2 * mu, :4, :4] = c * kappa * (np.eye(4) + g)
    return W


def series_weights(kappa):
    return [hopping_weights(kappa, 1.0, 4, 8), hopping_weights(kappa, 1j, 8, 8),
            hopping_weights(kappa, -1j, 8, 4)]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6), (4, 6, 2, 4)])
def test_network_with_series_weights_is_truncated_neumann_series(dims):
    kappa = 0.13
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=41)
    y = nn.network(b, U, series_weights(kappa), dims)
    want = b.copy()
    t = b
    for _ in range(3):
        t = kappa * oracle.hop(t, U, dims)
        want = want + t
    assert np.linalg.norm(y - want) / np.linalg.norm(want) < 1e-14


def test_single_layer_hopping_is_the_hopping_term():
    dims, kappa = (4, 4, 4, 8), 0.1
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=42)
    W = hopping_weights(kappa, 1.0, 4, 4)
    W[0] = 0
    assert np.allclose(nn.layer(b, U, W, dims), kappa * oracle.hop(b, U, dims), atol=1e-14)


def test_layer_gauge_covariance():
    dims = (4, 4, 2, 4)
    U = fields.su3_links(dims, workers=1)
    om = fields.gauge_transform(dims)
    r = np.random.default_rng(3)
    W = r.normal(size=(9, 8, 4)) + 1j * r.normal(size=(9, 8, 4))
    phi = r.normal(size=(fields.volume(dims), 4, 3)) + 1j * r.normal(size=(fields.volume(dims), 4, 3))
    lhs = nn.layer(np.einsum("xab,xcb->xca", om, phi), gauge_rotate(U, om, dims), W, dims)
    rhs = np.einsum("xab,xcb->xca", om, nn.layer(phi, U, W, dims))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-13


def test_adjoint_rule():
    dims = (4, 2, 4, 4)
    U = fields.su3_links(dims, workers=1)
    r = np.random.default_rng(5)
    W = r.normal(size=(9, 4, 8)) + 1j * r.normal(size=(9, 4, 8))
    V = fields.volume(dims)
    phi = r.normal(size=(V, 8, 3)) + 1j * r.normal(size=(V, 8, 3))
    psi = r.normal(size=(V, 4, 3)) + 1j * r.normal(size=(V, 4, 3))
    lhs = np.vdot(psi, nn.layer(phi, U, W, dims))
    rhs = np.vdot(nn.layer(psi, U, nn.adjoint_weights(W), dims), phi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_weight_vector_roundtrip():
    Ws = series_weights(0.12)
    flat = nn.join_weights(Ws)
    assert flat.size == 2304
    back = nn.split_weights(flat)
    for a, b in zip(Ws, back):
        assert np.allclose(a, b, atol=1e-7)
