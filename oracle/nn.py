"""FP64 numpy restatement of the learned preconditioner's layer (test
infrastructure only; shares nothing with the CUDA code).

    y(x)[o][a] = sum_{d=0..8} sum_i W_d[o][i] (T_d phi)(x)[i][a]
    T_0 phi(x) = phi(x)
    T_{1+2mu} phi(x) = s U_mu(x) phi(x + mu)
    T_{2+2mu} phi(x) = s U_mu(x - mu)^+ phi(x - mu)

with s = -1 on hops that cross the time boundary (the Wilson operator's
antiperiodic condition).  Fields are complex128[V, C, 3] in lexicographic site
order (for C = 4 this is the canonical spinor [V][spin][colour]); W is
complex128[9, C_out, C_in].

Parity unpinned by the paper (the paper has no such network).  Pinned in the
CPU tests by: (1) hopping-series weights built from the C oracle's gamma
matrices reproduce sum_{n<=3} (kappa H)^n of the C oracle's hopping term;
(2) gauge covariance; (3) the adjoint rule W'_e = W_{opp(e)}^+ used by
backpropagation.
"""
from __future__ import annotations

import numpy as np


def _coords(dims):
    L0, L1, L2, L3 = dims
    i = np.arange(L0 * L1 * L2 * L3)
    return np.stack([i % L0, (i // L0) % L1, (i // (L0 * L1)) % L2, i // (L0 * L1 * L2)], 1)


def _lex(x, dims):
    L0, L1, L2, _ = dims
    return x[:, 0] + L0 * (x[:, 1] + L1 * (x[:, 2] + L2 * x[:, 3]))


def transports(dims):
    """For d = 0..8: (neighbour index, link direction, link site, forward?, sign)."""
    x = _coords(dims)
    out = [(np.arange(len(x)), None, None, True, np.ones(len(x)))]
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % dims[mu]
        sgn = np.where((mu == 3) & (x[:, 3] == dims[3] - 1), -1.0, 1.0)
        out.append((_lex(y, dims), mu, np.arange(len(x)), True, sgn))
        y = x.copy()
        y[:, mu] = (y[:, mu] - 1) % dims[mu]
        sgn = np.where((mu == 3) & (x[:, 3] == 0), -1.0, 1.0)
        out.append((_lex(y, dims), mu, _lex(y, dims), False, sgn))
    return out


def transport(phi, U, dims, d, tr=None):
    tr = tr or transports(dims)
    nb, mu, lsite, fwd, sgn = tr[d]
    v = phi[nb]
    if mu is None:
        return v.copy()
    u = U[mu][lsite]
    if fwd:
        t = np.einsum("xab,xcb->xca", u, v)
    else:
        t = np.einsum("xba,xcb->xca", np.conj(u), v)
    return sgn[:, None, None] * t


def layer(phi, U, W, dims):
    tr = transports(dims)
    y = np.zeros((phi.shape[0], W.shape[1], 3), dtype=np.complex128)
    for d in range(9):
        y += np.einsum("oi,xia->xoa", W[d], transport(phi, U, dims, d, tr))
    return y


def network(b, U, Ws, dims):
    h = b
    for W in Ws:
        h = layer(h, U, W, dims)
    return h


def adjoint_weights(W):
    """W'_e = W_{opp(e)}^+ (opp exchanges the forward and backward hop of mu)."""
    opp = [0, 2, 1, 4, 3, 6, 5, 8, 7]
    return np.stack([np.conj(W[opp[e]]).T for e in range(9)])


def split_weights(flat):
    """The library's flat FP32 weight vector -> three complex [9, C_out, C_in]."""
    shapes = [(8, 4), (8, 8), (4, 8)]
    out, off = [], 0
    for co, ci in shapes:
        n = 9 * co * ci * 2
        w = np.asarray(flat[off:off + n], dtype=np.float64).reshape(9, co, ci, 2)
        out.append(w[..., 0] + 1j * w[..., 1])
        off += n
    return out


def join_weights(Ws):
    return np.concatenate([np.stack([W.real, W.imag], -1).reshape(-1) for W in Ws]).astype(
        np.float32)
