"""Flexible CG on the even-odd system with the network preconditioner
N_e N_e^+ (GPU), at kappa = 0.137: beyond the critical region of these links,
where GCR on D stalls.  Every solve is judged by the oracle's own true residual
||b - D x|| / ||b|| on the whole lattice (FP64, C oracle), computed from the
returned x.

* series weights (the truncated hopping series of D^-1), trained weights and
  no network (plain CGNR) each reach 1.05e-10 without the plain-CG fallback;
* the series preconditioner needs well under the iterations of the
  unpreconditioned even-odd CGNR (its even-even block is 1 + kappa^2 H_eo H_oe,
  the first Neumann term of Mhat^-1);
* the fallback: with maxiter = 3 the preconditioned iteration stops short and
  the even-odd CG finishes the solve from its iterate.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields

pytestmark = pytest.mark.gpu

KAPPA = 0.137
DIMS = (8, 8, 8, 16)


@pytest.fixture(scope="module")
def problem():
    U = fields.su3_links(DIMS, workers=1)
    b = fields.gaussian_spinor(DIMS, seed=2026)
    Ug = torch.from_numpy(U.view(np.float64).reshape(-1).copy()).cuda()
    bd = torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda()
    return U, b, Ug, bd


def true_residual(U, b, xd):
    x = xd.cpu().numpy().view(np.complex128).reshape(b.shape)
    return np.linalg.norm(b - oracle.apply_D(x, U, DIMS, KAPPA)) / np.linalg.norm(b)


def series_weights():
    w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
    W.wd_nn_init(w, KAPPA)
    return w


def test_fcg_series_trained_and_plain(problem):
    U, b, Ug, bd = problem
    trained = series_weights()
    p = W.wd_nn_train_params_default()
    p.samples, p.batch = 256, 8
    W.wd_nn_train(trained, Ug, KAPPA, DIMS, p)
    iters = {}
    for name, wts in (("series", series_weights()), ("trained", trained), ("plain", None)):
        x = torch.zeros_like(bd)
        info = W.wd_solve_fcg(x, bd, Ug, KAPPA, DIMS, wts)
        assert info["fallback_iters"] == 0, (name, info)
        r = true_residual(U, b, x)
        assert r <= 1.05e-10, (name, r, info)
        assert abs(r - info["true_residual"]) <= 1e-11, (name, r, info)
        iters[name] = info["iters"]
    assert iters["series"] < 0.7 * iters["plain"], iters


def test_fcg_falls_back_to_plain_cg(problem):
    U, b, Ug, bd = problem
    x = torch.zeros_like(bd)
    q = W.wd_solve_params_default()
    q.maxiter = 3
    info = W.wd_solve_fcg(x, bd, Ug, KAPPA, DIMS, series_weights(), q)
    assert info["fallback_iters"] > 0, info
    assert true_residual(U, b, x) <= 1.05e-10


def test_fcg_host_buffers(problem):
    """x and b in host memory (staged by the library), series preconditioner"""
    U, b, _, _ = problem
    x = np.zeros_like(b)
    info = W.wd_solve_fcg(x, b, U, KAPPA, DIMS, series_weights())
    assert info["fallback_iters"] == 0
    r = np.linalg.norm(b - oracle.apply_D(x, U, DIMS, KAPPA)) / np.linalg.norm(b)
    assert r <= 1.05e-10, r
