"""Solver tests (GPU): wd_solve / wd_solve_ex reach the requested true
residual ||b - D x|| / ||b||, measured independently by the FP64 oracle on
the unpacked solution, for every inner precision; plus the degenerate and
failure cases, all made on the host (bad inputs, tiny iteration caps)."""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import dev

pytestmark = pytest.mark.gpu


def true_residual(x, b, U, dims, kappa):
    r = b - oracle.apply_D(x, U, dims, kappa)
    return np.linalg.norm(r) / np.linalg.norm(b)


def params(**kw):
    p = W.wd_solve_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.12), ((4, 4, 4, 8), 0.137),
                                        ((6, 6, 6, 6), 0.135), ((8, 8, 8, 8), 0.137)])
@pytest.mark.parametrize("inner", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_solve_reaches_tolerance(dims, kappa, inner):
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=2024)
    x = np.zeros_like(b)
    info = W.wd_solve_ex(x, b, U, kappa, dims, params(inner_prec=inner))
    assert info["status"] == W.WD_OK
    assert info["true_residual"] <= 1e-10
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10


def test_wd_solve_default_entry_point_device_pointers():
    dims, kappa = (4, 6, 8, 10), 0.13
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=7)
    xd = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
    W.wd_solve(xd, dev(b), dev(U), kappa, 1e-10, dims)
    x = xd.cpu().numpy().view(np.complex128).reshape(b.shape)
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10


def test_graph_and_plain_launches_agree_bitwise():
    dims, kappa = (4, 4, 4, 8), 0.137
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=5)
    x1 = np.zeros_like(b)
    x2 = np.zeros_like(b)
    i1 = W.wd_solve_ex(x1, b, U, kappa, dims, params(use_graph=1))
    i2 = W.wd_solve_ex(x2, b, U, kappa, dims, params(use_graph=0))
    assert i1["iters"] == i2["iters"]
    assert np.array_equal(x1, x2)


def test_point_source_and_zero_rhs():
    dims, kappa = (4, 4, 4, 4), 0.12
    U = fields.su3_links(dims, workers=1)
    b = fields.point_source(dims, 0, 2, 1)
    x = np.zeros_like(b)
    W.wd_solve_ex(x, b, U, kappa, dims, params(inner_prec=W.WD_F16))
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10
    z = np.zeros_like(b)
    xz = np.ones_like(b)
    info = W.wd_solve_ex(xz, z, U, kappa, dims)
    assert info["status"] == W.WD_OK and np.all(xz == 0)


def test_initial_guess_resume():
    dims, kappa = (4, 4, 4, 8), 0.137
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=11)
    x = np.zeros_like(b)
    first = W.wd_solve_ex(x, b, U, kappa, dims, params(tol=1e-6))
    assert first["status"] == W.WD_OK
    again = W.wd_solve_ex(x, b, U, kappa, dims, params(use_initial_guess=1))
    assert again["status"] == W.WD_OK
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10
    fresh = W.wd_solve_ex(np.zeros_like(b), b, U, kappa, dims, params())
    assert again["iters"] < fresh["iters"]


def test_maxiter_reports_noconv_with_best_iterate():
    dims, kappa = (4, 4, 4, 8), 0.137
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=12)
    x = np.zeros_like(b)
    info = W.wd_solve_ex(x, b, U, kappa, dims, params(maxiter=4), check=False)
    assert info["status"] == W.WD_ERR_NOCONV
    r = true_residual(x, b, U, dims, kappa)
    assert r < 1.0 and abs(r - info["true_residual"]) < 1e-12


def test_nonfinite_rhs_detected():
    dims, kappa = (4, 4, 4, 4), 0.12
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=13)
    b[17, 1, 2] = np.nan
    info = W.wd_solve_ex(np.zeros_like(b), b, U, kappa, dims, check=False)
    assert info["status"] == W.WD_ERR_NONFINITE


def test_bad_solver_params():
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims)
    info = W.wd_solve_ex(np.zeros_like(b), b, U, 0.12, dims, params(inner_prec=W.WD_F16,
                                                                     inner_recon=18), check=False)
    assert info["status"] == W.WD_ERR_PREC
    info = W.wd_solve_ex(np.zeros_like(b), b, U, 0.12, dims, params(tol=-1.0), check=False)
    assert info["status"] == W.WD_ERR_ARG


@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.12), ((4, 4, 4, 8), 0.137),
                                        ((6, 6, 6, 6), 0.135), ((8, 8, 8, 8), 0.137)])
@pytest.mark.parametrize("inner", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_bicgstab_reaches_tolerance(dims, kappa, inner):
    """BiCGstab on the Schur operator (the paper's second inverter), with the
    same FP64 reliable updates; judged by the oracle's true residual."""
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=2024)
    x = np.zeros_like(b)
    info = W.wd_solve_ex(x, b, U, kappa, dims, params(inner_prec=inner,
                                                      solver=W.WD_SOLVER_BICGSTAB))
    assert info["status"] == W.WD_OK
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10


def test_bicgstab_in_temporal_gauge_and_plain_launches():
    dims, kappa = (4, 6, 8, 10), 0.13
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=31)
    for gf, graph in ((1, 1), (0, 0)):
        x = np.zeros_like(b)
        W.wd_solve_ex(x, b, U, kappa, dims, params(solver=W.WD_SOLVER_BICGSTAB, gauge_fix=gf,
                                                   use_graph=graph))
        assert true_residual(x, b, U, dims, kappa) <= 1.05e-10


def test_batch_rejects_bicgstab():
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims)[None]
    rc, _ = W.wd_solve_batch([{"dims": dims, "kappa": 0.12, "nrhs": 1, "gauge": U, "b": b,
                               "x": np.zeros_like(b)}], params(solver=W.WD_SOLVER_BICGSTAB),
                             check=False)
    assert rc == W.WD_ERR_ARG


@pytest.mark.parametrize("solver,gf", [(W.WD_SOLVER_CG, 1), (W.WD_SOLVER_BICGSTAB, 0),
                                       (W.WD_SOLVER_BICGSTAB, 1)])
def test_initial_guess_resume_other_variants(solver, gf):
    """A solve restarted from a partial solution (the FP64 residual of a
    nonzero x is formed in setup) reaches the tolerance, in temporal gauge and
    with BiCGstab too, in fewer iterations than a start from zero."""
    dims, kappa = (4, 4, 4, 8), 0.128
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=12)
    x = np.zeros_like(b)
    first = W.wd_solve_ex(x, b, U, kappa, dims, params(tol=1e-5, solver=solver, gauge_fix=gf))
    assert first["status"] == W.WD_OK
    again = W.wd_solve_ex(x, b, U, kappa, dims,
                          params(use_initial_guess=1, solver=solver, gauge_fix=gf))
    assert again["status"] == W.WD_OK
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10
    fresh = W.wd_solve_ex(np.zeros_like(b), b, U, kappa, dims,
                          params(solver=solver, gauge_fix=gf))
    assert again["iters"] < fresh["iters"]


@pytest.mark.parametrize("reliable,check", [(1, 2), (7, 3), (50, 16), (3, 1)])
@pytest.mark.parametrize("inner", [W.WD_F32, W.WD_F16])
def test_solver_schedule_edges(reliable, check, inner):
    """Reliable updates every iteration or at odd intervals, and check
    intervals that are odd, 1 or long (the graph chunk rounds to an even
    count of at least 2): every schedule reaches the oracle's 1e-10."""
    dims, kappa = (4, 4, 4, 8), 0.132
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=13)
    x = np.zeros_like(b)
    info = W.wd_solve_ex(x, b, U, kappa, dims,
                         params(inner_prec=inner, reliable_interval=reliable,
                                check_interval=check))
    assert info["status"] == W.WD_OK
    assert true_residual(x, b, U, dims, kappa) <= 1.05e-10
