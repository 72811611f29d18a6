"""Parity of libwd's hopping kernels with the FP64 oracle (GPU).

Each case runs the CUDA kernel through the C ABI on seeded synthetic fields
and compares every output component with the oracle's.  Tolerances (relative
l2 error, and largest elementwise error relative to the largest reference
magnitude): FP64 1e-13, FP32 1e-6, FP16 with per-site scale 5e-3.
Lattices span the degenerate 2-site extent, several thread blocks, ragged
tails (Vh not a multiple of the 32-site block or of the 128-thread CTA) and
an irregular shape.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import (NORM_TOL, PREC_TOL, dev, host, pack_gauge, pack_spinor, rel_l2,
                           rel_max, unpack_spinor)

pytestmark = pytest.mark.gpu

DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 4, 4, 8), (6, 6, 6, 6), (4, 6, 8, 10), (8, 8, 8, 8),
        (2, 4, 2, 6)]
FORMATS = [(W.WD_F64, 18), (W.WD_F64, 12), (W.WD_F32, 18), (W.WD_F32, 12), (W.WD_F16, 12)]

_cache = {}


def field(dims):
    if dims not in _cache:
        _cache[dims] = (fields.su3_links(dims, workers=1), fields.gaussian_spinor(dims))
    return _cache[dims]


def check(got, want, prec):
    tol = PREC_TOL[prec]
    assert rel_l2(got, want) <= tol, rel_l2(got, want)
    assert rel_max(got, want) <= 4 * tol, rel_max(got, want)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,recon", FORMATS)
@pytest.mark.parametrize("dagger", [0, 1])
def test_hop_block_matches_oracle(dims, prec, recon, dagger):
    U, psi = field(dims)
    g = pack_gauge(U, dims, prec, recon)
    for p in (W.WD_EVEN, W.WD_ODD):
        src = oracle.restrict(psi, dims, 1 - p)
        inp = pack_spinor(src, dims, 1 - p, prec)
        out = W.alloc_spinor(dims, p, prec)
        W.wd_dslash_ex(out, inp, g, p, dagger, 1.0, None, 0.0, None, 0.0, None, dims, prec, recon)
        got = unpack_spinor(out, dims, p, prec)
        want = oracle.hop_block(p, src, U, dims, dagger=bool(dagger))
        check(got, want, prec)


@pytest.mark.parametrize("prec", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_full_operator_config_4x4(prec):
    """D psi on 4^4, kappa = 0.12 (the full-lattice operator), both D and D^+."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U, psi = field(dims)
    g = pack_gauge(U, dims, prec, 12)
    inp = pack_spinor(psi, dims, W.WD_FULL, prec)
    out = W.alloc_spinor(dims, W.WD_FULL, prec)
    W.wd_dslash(out, inp, g, kappa, W.WD_FULL, dims, prec)
    check(unpack_spinor(out, dims, W.WD_FULL, prec), oracle.apply_D(psi, U, dims, kappa), prec)
    W.wd_dslash_dag(out, inp, g, kappa, W.WD_FULL, dims, prec)
    check(unpack_spinor(out, dims, W.WD_FULL, prec),
          oracle.apply_D(psi, U, dims, kappa, dagger=True), prec)


@pytest.mark.parametrize("prec", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_parity_dslash_scaled_by_minus_kappa(prec):
    dims, kappa = (4, 6, 8, 10), 0.1365
    U, psi = field(dims)
    g = pack_gauge(U, dims, prec, 12)
    src = oracle.restrict(psi, dims, 1)
    inp = pack_spinor(src, dims, 1, prec)
    out = W.alloc_spinor(dims, 0, prec)
    W.wd_dslash(out, inp, g, kappa, W.WD_EVEN, dims, prec)
    check(unpack_spinor(out, dims, 0, prec), -kappa * oracle.hop_block(0, src, U, dims), prec)


@pytest.mark.parametrize("prec", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_epilogue_xpay_and_norm(prec):
    """out = a H in + bx x + cy y with ||out||^2, x aliasing out."""
    dims = (6, 6, 6, 6)
    U, psi = field(dims)
    g = pack_gauge(U, dims, prec, 12)
    src = oracle.restrict(psi, dims, 0)
    xh = fields.gaussian_spinor(dims, seed=77)[: len(src)]
    yh = fields.gaussian_spinor(dims, seed=78)[: len(src)]
    inp = pack_spinor(src, dims, 0, prec)
    xb = pack_spinor(xh, dims, 1, prec)
    yb = pack_spinor(yh, dims, 1, prec)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    a, bx, cy = -0.137 ** 2, 0.75, -1.25
    W.wd_dslash_ex(xb, inp, g, 1, 0, a, xb, bx, yb, cy, nrm, dims, prec, 12)
    got = unpack_spinor(xb, dims, 1, prec)
    want = a * oracle.hop_block(1, src, U, dims) + bx * xh + cy * yh
    check(got, want, prec)
    # the reported norm is the norm of the stored field
    assert abs(nrm.item() - np.vdot(got, got).real) <= NORM_TOL[prec] * np.vdot(got, got).real


@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F16, 12)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_schur_operator(prec, recon, dagger):
    dims, kappa = (4, 4, 4, 8), 0.137
    U, psi = field(dims)
    g = pack_gauge(U, dims, prec, recon)
    xe = oracle.restrict(psi, dims, 0)
    inp = pack_spinor(xe, dims, 0, prec)
    out = W.alloc_spinor(dims, 0, prec)
    tmp = W.alloc_spinor(dims, 1, prec)
    W.wd_mhat(out, inp, g, tmp, kappa, dagger, dims, prec, recon)
    check(unpack_spinor(out, dims, 0, prec), oracle.schur(xe, U, dims, kappa, bool(dagger)), prec)


def test_unit_links_free_field_gpu():
    """With unit links a plane wave is an eigenvector (cross-check of the
    antiperiodic boundary on the GPU path, independent of random links)."""
    dims, kappa = (4, 4, 4, 8), 0.12
    x = fields.coords(dims)
    p = np.array([np.pi / 2, np.pi, 3 * np.pi / 2, 3 * np.pi / 8])
    chi = np.arange(12).reshape(4, 3) + 1j
    psi = np.exp(1j * (x @ p))[:, None, None] * chi[None]
    U = fields.unit_links(dims)
    g = pack_gauge(U, dims, W.WD_F64, 12)
    inp = pack_spinor(psi, dims, W.WD_FULL, W.WD_F64)
    out = W.alloc_spinor(dims, W.WD_FULL, W.WD_F64)
    W.wd_dslash(out, inp, g, kappa, W.WD_FULL, dims, W.WD_F64)
    check(unpack_spinor(out, dims, W.WD_FULL, W.WD_F64), oracle.apply_D(psi, U, dims, kappa),
          W.WD_F64)


@pytest.mark.parametrize("prec", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_pack_unpack_roundtrip(prec):
    dims = (6, 6, 6, 6)
    _, psi = field(dims)
    buf = pack_spinor(psi, dims, W.WD_FULL, prec)
    back = unpack_spinor(buf, dims, W.WD_FULL, prec)
    if prec == W.WD_F64:
        assert np.array_equal(back, psi)
    elif prec == W.WD_F32:
        assert np.array_equal(back, psi.astype(np.complex64).astype(np.complex128))
    else:
        # half with a per-site scale: |error| <= 2^-11 * site max-abs (round to nearest)
        site_max = np.max(np.maximum(np.abs(psi.real), np.abs(psi.imag)), axis=(1, 2))
        err = np.max(np.maximum(np.abs((back - psi).real), np.abs((back - psi).imag)), axis=(1, 2))
        assert np.all(err <= site_max * 2.0 ** -11 * 1.001)


@pytest.mark.parametrize("prec", [W.WD_F64, W.WD_F32, W.WD_F16])
def test_blas_reductions(prec):
    dims = (4, 6, 8, 10)
    _, psi = field(dims)
    a_h = oracle.restrict(psi, dims, 0)
    b_h = fields.gaussian_spinor(dims, seed=99)[: len(a_h)]
    A = pack_spinor(a_h, dims, 0, prec)
    B = pack_spinor(b_h, dims, 0, prec)
    a_q = unpack_spinor(A, dims, 0, prec)   # the values actually stored
    b_q = unpack_spinor(B, dims, 0, prec)
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    W.wd_norm2(res, A, dims, 0, prec)
    assert abs(res[0].item() - np.vdot(a_q, a_q).real) <= NORM_TOL[prec] * np.vdot(a_q, a_q).real
    W.wd_cdot(res, A, B, dims, 0, prec)
    z = np.vdot(a_q, b_q)
    got = complex(res[0].item(), res[1].item())
    assert abs(got - z) <= NORM_TOL[prec] * np.linalg.norm(a_q) * np.linalg.norm(b_q)
    W.wd_axpby(0.5, A, -2.0, B, dims, 0, prec)
    check(unpack_spinor(B, dims, 0, prec), 0.5 * a_q - 2.0 * b_q, prec)


def test_reduction_is_deterministic():
    dims = (8, 8, 8, 8)
    _, psi = field(dims)
    A = pack_spinor(psi, dims, W.WD_FULL, W.WD_F32)
    res = torch.zeros(8, dtype=torch.float64, device="cuda")
    for k in range(8):
        W.wd_norm2(res[k:k + 1], A, dims, W.WD_FULL, W.WD_F32)
    r = res.cpu().numpy()
    assert np.all(r == r[0])


def test_convert_precisions():
    dims = (4, 4, 4, 4)
    _, psi = field(dims)
    A = pack_spinor(psi, dims, W.WD_FULL, W.WD_F64)
    B = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    W.wd_convert_spinor(B, W.WD_F32, A, W.WD_F64, dims, W.WD_FULL)
    got = unpack_spinor(B, dims, W.WD_FULL, W.WD_F32)
    assert np.array_equal(got, psi.astype(np.complex64).astype(np.complex128))


@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F16, 12)])
@pytest.mark.parametrize("flags", [0, W.WD_TEMPORAL_GAUGE])
def test_every_cta_size_is_bit_identical(prec, recon, flags):
    """The CTA sizes the single-field autotuner may choose (64, 128, 256
    sites) give bit-identical fields, H and H^+, with the fused epilogue, on
    a lattice whose last CTA is ragged for every size; and they match the
    oracle.  Temporal-gauge links come from the host definition."""
    from tests._wdutil import temporal_gauge_links
    dims = (6, 4, 6, 10)   # V/2 = 720 sites: 11.25, 5.6, 2.8 CTAs
    U = fields.su3_links(dims, workers=1)
    if flags:
        U, _ = temporal_gauge_links(U, dims)
    g = pack_gauge(U, dims, prec, recon)
    psi = fields.gaussian_spinor(dims)
    xh = fields.to_half(fields.gaussian_spinor(dims, seed=91), dims, 0)
    src = fields.to_half(psi, dims, 1)
    inp = pack_spinor(src, dims, 1, prec)
    xb = pack_spinor(xh, dims, 0, prec)
    try:
        for dagger in (0, 1):
            outs = {}
            for bs in (128, 64, 256):
                W.wd_dslash_set_block(bs)
                out = W.alloc_spinor(dims, 0, prec)
                W.wd_dslash_ex(out, inp, g, 0, dagger, -0.13, xb, 0.5, None, 0.0, None, dims,
                               prec, recon | flags)
                torch.cuda.synchronize()
                outs[bs] = unpack_spinor(out, dims, 0, prec)
            assert np.array_equal(outs[64], outs[128]) and np.array_equal(outs[256], outs[128])
            want = -0.13 * oracle.hop_block(0, src, U, dims, dagger=bool(dagger)) + 0.5 * xh
            assert rel_l2(outs[128], want) <= PREC_TOL[prec]
    finally:
        W.wd_dslash_set_block(0)


def test_cta_size_tuner_reports_its_choice():
    dims = (8, 6, 4, 12)   # a shape no other test uses
    prev = W.wd_set_autotune(1)
    try:
        U = fields.su3_links(dims, workers=1)
        g = pack_gauge(U, dims, W.WD_F32, 12)
        inp = pack_spinor(fields.to_half(fields.gaussian_spinor(dims), dims, 1), dims, 1,
                          W.WD_F32)
        out = W.alloc_spinor(dims, 0, W.WD_F32)
        W.wd_dslash(out, inp, g, 0.13, 0, dims, W.WD_F32)
        torch.cuda.synchronize()
    finally:
        W.wd_set_autotune(prev)
    _, text = W.wd_tune_report()
    mine = [l for l in text.splitlines() if l.startswith("dslash prec=1 recon=12 dagger=0 tg=0")
            and "dims=8x6x4x12 " in l]
    assert len(mine) == 1, text
    us = [float(v) for v in mine[0].split("us[64,128,256]=")[1].split()[0].split(",")]
    block = int(mine[0].split("block=")[1])
    assert all(v > 0 for v in us) and us[[64, 128, 256].index(block)] == min(us)
    # the choice changes nothing in the result
    want = -0.13 * oracle.hop_block(0, fields.to_half(fields.gaussian_spinor(dims), dims, 1), U,
                                    dims)
    assert rel_l2(unpack_spinor(out, dims, 0, W.WD_F32), want) <= PREC_TOL[W.WD_F32]


def test_cta_size_rejects_other_values():
    for bad in (32, 96, 512):
        with pytest.raises(W.WdError):
            W.wd_dslash_set_block(bad)


@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F16, 12)])
def test_launch_overlap_chain_is_bit_identical(prec, recon):
    """A chain of dependent hopping launches (each reads the field the
    previous one wrote, alternating parity, plain and with the fused norm) as
    programmatic dependent launches gives exactly the fields and norms of
    plain stream-ordered launches; and the two-hop result matches the
    oracle."""
    dims = (8, 6, 4, 12)
    U, psi = fields.su3_links(dims, workers=1), fields.gaussian_spinor(dims)
    g = pack_gauge(U, dims, prec, recon)
    src = fields.to_half(psi, dims, 1)
    res = {}
    prev = W.wd_set_launch_overlap(1)
    try:
        for on in (1, 0):
            W.wd_set_launch_overlap(on)
            a = pack_spinor(src, dims, 1, prec)
            b = W.alloc_spinor(dims, 0, prec)
            nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
            for _ in range(5):   # a -> b (even), b -> a (odd), ...
                W.wd_dslash_ex(b, a, g, 0, 0, -0.12, None, 0.0, None, 0.0, None, dims, prec,
                               recon)
                W.wd_dslash_ex(a, b, g, 1, 0, -0.12, None, 0.0, None, 0.0, nrm, dims, prec,
                               recon)
            torch.cuda.synchronize()
            res[on] = (unpack_spinor(a, dims, 1, prec), unpack_spinor(b, dims, 0, prec),
                       float(nrm.item()))
    finally:
        W.wd_set_launch_overlap(prev)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]
    # one more pair from the chain's last odd field, checked against the oracle
    odd = res[1][0]
    want_b = -0.12 * oracle.hop_block(0, odd, U, dims)
    a = pack_spinor(odd, dims, 1, prec)
    b = W.alloc_spinor(dims, 0, prec)
    W.wd_dslash_ex(b, a, g, 0, 0, -0.12, None, 0.0, None, 0.0, None, dims, prec, recon)
    torch.cuda.synchronize()
    assert rel_l2(unpack_spinor(b, dims, 0, prec), want_b) <= PREC_TOL[prec]


def test_launch_overlap_solve_is_bit_identical():
    """The mixed-precision solve (graphs of hopping and BLAS launches) gives
    the same iterate, iteration count and residual with and without launch
    overlap, and the oracle confirms the residual."""
    dims, kappa = (8, 8, 8, 8), 0.137
    U, b = fields.su3_links(dims, workers=1), fields.gaussian_spinor(dims, seed=7)
    out = {}
    prev = W.wd_set_launch_overlap(1)
    try:
        for on in (1, 0):
            W.wd_set_launch_overlap(on)
            x = np.zeros_like(b)
            q = W.wd_solve_params_default()
            q.inner_prec = W.WD_F16
            info = W.wd_solve_ex(x, b, U, kappa, dims, q)
            out[on] = (x, info["iters"], info["true_residual"])
    finally:
        W.wd_set_launch_overlap(prev)
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]
    r = b - oracle.apply_D(out[1][0], U, dims, kappa)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.05e-10
