"""Temporal gauge (the paper's gauge-fixing trick) on the GPU, against numpy
and the FP64 oracle.

* the transformation: U'_t = 1 off the last time slice, U' = omega U
  omega^+ (numpy, independent of the GPU kernel), omega unitary;
* the hopping kernels with WD_TEMPORAL_GAUGE skip the identity time links and
  still match the oracle applied to U';
* the full-operator covariance D[U'] (omega psi) = omega D[U] psi;
* a solve with gauge_fix = 1 reaches 1e-10 on the ORIGINAL system.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import (PREC_TOL, dev, host, pack_gauge, pack_spinor, rel_l2, rel_max,
                           unpack_spinor)
from tests.test_oracle_pins import gauge_rotate
from tests._wdutil import temporal_gauge_links

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 8), (6, 4, 2, 6), (2, 2, 2, 2)]


def fix(U, dims):
    V = fields.volume(dims)
    Uo = torch.empty(4 * V * 18, dtype=torch.float64, device="cuda")
    om = torch.empty(V * 18, dtype=torch.float64, device="cuda")
    W.wd_gauge_fix_temporal(Uo, om, dev(U), dims)
    return host(Uo, (4, V, 3, 3)), host(om, (V, 3, 3))


@pytest.mark.parametrize("dims", DIMS)
def test_temporal_gauge_transformation(dims):
    U = fields.su3_links(dims, workers=1)
    Up, om = fix(U, dims)
    x = fields.coords(dims)
    inner = x[:, 3] < dims[3] - 1
    eye = np.eye(3)
    assert np.max(np.abs(Up[3][inner] - eye)) == 0.0
    assert np.max(np.abs(np.conj(np.swapaxes(om, 1, 2)) @ om - eye)) < 1e-13
    # omega from its definition, by a plain cumulative product along t
    S = dims[0] * dims[1] * dims[2]
    om_np = np.zeros_like(om)
    om_np[:S] = eye
    for t in range(dims[3] - 1):
        sl = slice(t * S, (t + 1) * S)
        om_np[(t + 1) * S:(t + 2) * S] = om_np[sl] @ U[3][sl]
    assert np.max(np.abs(om - om_np)) < 1e-13
    want = gauge_rotate(U, om_np, dims)
    mask = np.ones(want.shape[:2], bool)
    mask[3][inner] = False   # the kernel writes those exactly as the identity
    assert np.max(np.abs(Up[mask] - want[mask])) < 1e-13


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F16, 12)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_temporal_gauge_dslash(dims, prec, recon, dagger):
    # the oracle's links come from the host definition, not from the GPU
    U = fields.su3_links(dims, workers=1)
    Up, _ = temporal_gauge_links(U, dims)
    psi = fields.gaussian_spinor(dims)
    g = pack_gauge(Up, dims, prec, recon)
    for p in (0, 1):
        src = oracle.restrict(psi, dims, 1 - p)
        inp = pack_spinor(src, dims, 1 - p, prec)
        out = W.alloc_spinor(dims, p, prec)
        W.wd_dslash_ex(out, inp, g, p, dagger, 1.0, None, 0.0, None, 0.0, None, dims, prec,
                       recon | W.WD_TEMPORAL_GAUGE)
        got = unpack_spinor(out, dims, p, prec)
        want = oracle.hop_block(p, src, Up, dims, dagger=bool(dagger))
        assert rel_l2(got, want) <= PREC_TOL[prec]
        assert rel_max(got, want) <= 4 * PREC_TOL[prec]


def test_temporal_gauge_covariance_full_operator():
    dims, kappa = (4, 4, 4, 8), 0.12
    U = fields.su3_links(dims, workers=1)
    Up, om = temporal_gauge_links(U, dims)
    psi = fields.gaussian_spinor(dims)
    g = pack_gauge(Up, dims, W.WD_F64, 18)
    rot = np.einsum("xab,xsb->xsa", om, psi)
    inp = pack_spinor(rot, dims, W.WD_FULL, W.WD_F64)
    out = W.alloc_spinor(dims, W.WD_FULL, W.WD_F64)
    h = W.wd_spinor_bytes(dims, 0, W.WD_F64)
    W.wd_dslash_ex(out[:h], inp[h:], g, 0, 0, -kappa, inp[:h], 1.0, None, 0.0, None, dims,
                   W.WD_F64, 18 | W.WD_TEMPORAL_GAUGE)
    W.wd_dslash_ex(out[h:], inp[:h], g, 1, 0, -kappa, inp[h:], 1.0, None, 0.0, None, dims,
                   W.WD_F64, 18 | W.WD_TEMPORAL_GAUGE)
    got = unpack_spinor(out, dims, W.WD_FULL, W.WD_F64)
    want = np.einsum("xab,xsb->xsa", om, oracle.apply_D(psi, U, dims, kappa))
    assert rel_l2(got, want) <= 1e-13


def test_rotate_spinor_roundtrip():
    dims = (4, 4, 4, 8)
    U = fields.su3_links(dims, workers=1)
    _, om = fix(U, dims)
    psi = fields.gaussian_spinor(dims)
    a = dev(psi)
    b = torch.empty_like(a)
    W.wd_rotate_spinor(b, a, dev(om), dims, 0)
    assert rel_l2(host(b, psi.shape), np.einsum("xab,xsb->xsa", om, psi)) <= 1e-15
    W.wd_rotate_spinor(b, b, dev(om), dims, 1)
    assert rel_l2(host(b, psi.shape), psi) <= 1e-14


@pytest.mark.parametrize("inner", [W.WD_F32, W.WD_F16, W.WD_F64])
def test_solve_in_temporal_gauge(inner):
    dims, kappa = (4, 4, 4, 8), 0.137
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=21)
    x = np.zeros_like(b)
    p = W.wd_solve_params_default()
    p.inner_prec = inner
    p.gauge_fix = 1
    info = W.wd_solve_ex(x, b, U, kappa, dims, p)
    assert info["status"] == W.WD_OK
    r = np.linalg.norm(b - oracle.apply_D(x, U, dims, kappa)) / np.linalg.norm(b)
    assert r <= 1.05e-10
