"""The FP16 hopping kernel with its far (z, t) neighbours staged in shared
memory by bulk asynchronous copies (GPU), against the oracle and against the
unstaged FP16 kernel.

Both kernels apply the same operations to every site in the same order (the
staging changes where the z and t neighbour spinors are read from, not what
is computed), so their outputs are compared bit for bit.  The lattices cover
the periodic wrap of the staged block index in z and t (extents 2 and 4),
slices of exactly one and of several 32-site blocks, a ragged last CTA, and
both parities, H and H^+, with the fused epilogue (x aliasing out, y)."""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import PREC_TOL, pack_gauge, pack_spinor, rel_l2, rel_max, unpack_spinor

pytestmark = pytest.mark.gpu

F16 = W.WD_F16
STAGED = 12 | W.WD_STAGE_NEIGHBOURS
# (L0 L1 / 2) % 32 == 0 in every shape: slices of 32, 64 and 288 sites
DIMS = [(8, 8, 2, 2), (4, 16, 4, 4), (8, 8, 6, 4), (24, 24, 2, 4), (16, 8, 4, 6)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [0, 1])
def test_staged_matches_unstaged_and_oracle(dims, dagger):
    U = fields.su3_links(dims, workers=1)
    psi = fields.gaussian_spinor(dims)
    g = pack_gauge(U, dims, F16, 12)
    for p in (W.WD_EVEN, W.WD_ODD):
        src = oracle.restrict(psi, dims, 1 - p)
        inp = pack_spinor(src, dims, 1 - p, F16)
        ref = W.alloc_spinor(dims, p, F16)
        out = W.alloc_spinor(dims, p, F16)
        W.wd_dslash_ex(ref, inp, g, p, dagger, 1.0, None, 0.0, None, 0.0, None, dims, F16, 12)
        W.wd_dslash_ex(out, inp, g, p, dagger, 1.0, None, 0.0, None, 0.0, None, dims, F16,
                       STAGED)
        torch.cuda.synchronize()
        got = unpack_spinor(out, dims, p, F16)
        assert np.array_equal(got, unpack_spinor(ref, dims, p, F16))
        want = oracle.hop_block(p, src, U, dims, dagger=bool(dagger))
        assert rel_l2(got, want) <= PREC_TOL[F16]
        assert rel_max(got, want) <= 4 * PREC_TOL[F16]


def test_staged_epilogue_with_aliasing():
    """out = a H in + bx x + cy y with x aliasing out, staged and unstaged."""
    dims = (8, 8, 6, 4)
    U = fields.su3_links(dims, workers=1)
    g = pack_gauge(U, dims, F16, 12)
    src = oracle.restrict(fields.gaussian_spinor(dims), dims, 0)
    xh = fields.gaussian_spinor(dims, seed=77)[: len(src)]
    yh = fields.gaussian_spinor(dims, seed=78)[: len(src)]
    inp = pack_spinor(src, dims, 0, F16)
    yb = pack_spinor(yh, dims, 1, F16)
    a, bx, cy = -0.137 ** 2, 0.75, -1.25
    res = []
    for recon in (12, STAGED):
        xb = pack_spinor(xh, dims, 1, F16)
        W.wd_dslash_ex(xb, inp, g, 1, 0, a, xb, bx, yb, cy, None, dims, F16, recon)
        torch.cuda.synchronize()
        res.append(unpack_spinor(xb, dims, 1, F16))
    assert np.array_equal(res[0], res[1])
    want = a * oracle.hop_block(1, src, U, dims) + bx * xh + cy * yh
    assert rel_l2(res[1], want) <= PREC_TOL[F16]


@pytest.mark.parametrize("case", ["dims", "prec", "norm", "gauge"])
def test_staged_rejects_what_it_does_not_cover(case):
    dims = (6, 6, 6, 6) if case == "dims" else (8, 8, 2, 2)  # (6, 6): 18-site slices
    prec = W.WD_F32 if case == "prec" else F16
    U = fields.su3_links(dims, workers=1)
    g = pack_gauge(U, dims, prec, 12)
    inp = W.alloc_spinor(dims, 1, prec)
    out = W.alloc_spinor(dims, 0, prec)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda") if case == "norm" else None
    recon = STAGED | (W.WD_TEMPORAL_GAUGE if case == "gauge" else 0)
    with pytest.raises(W.WdError):
        W.wd_dslash_ex(out, inp, g, 0, 0, 1.0, None, 0.0, None, 0.0, nrm, dims, prec, recon)


def test_staged_wait_timeout_is_reported_and_recoverable():
    """The failure path of the staged kernel's bounded wait, run on purpose
    and without any fault: with a wait limit of 0 polls every warp gives up
    at once, drains its copies with the long second wait, writes NaN and
    raises the device flag; wd_async_status reports WD_ERR_TIMEOUT once and
    clears it, and the next launch with the default limit is exact."""
    dims = (8, 8, 6, 4)
    U = fields.su3_links(dims, workers=1)
    psi = fields.gaussian_spinor(dims)
    g = pack_gauge(U, dims, F16, 12)
    src = oracle.restrict(psi, dims, 1)
    inp = pack_spinor(src, dims, 1, F16)
    ref = W.alloc_spinor(dims, 0, F16)
    W.wd_dslash_ex(ref, inp, g, 0, 0, 1.0, None, 0.0, None, 0.0, None, dims, F16, 12)
    want = unpack_spinor(ref, dims, 0, F16)
    assert W.wd_async_status() == W.WD_OK
    out = W.alloc_spinor(dims, 0, F16)
    try:
        W.wd_set_wait_limit(0)
        W.wd_dslash_ex(out, inp, g, 0, 0, 1.0, None, 0.0, None, 0.0, None, dims, F16, STAGED)
        assert W.wd_async_status() == W.WD_ERR_TIMEOUT
    finally:
        W.wd_set_wait_limit(1 << 22)
    torch.cuda.synchronize()
    assert np.all(np.isnan(unpack_spinor(out, dims, 0, F16).real))
    assert W.wd_async_status() == W.WD_OK  # cleared on read
    W.wd_dslash_ex(out, inp, g, 0, 0, 1.0, None, 0.0, None, 0.0, None, dims, F16, STAGED)
    assert W.wd_async_status() == W.WD_OK
    assert np.array_equal(unpack_spinor(out, dims, 0, F16), want)


def test_wait_limit_range():
    with pytest.raises(W.WdError):
        W.wd_set_wait_limit(-1)
    with pytest.raises(W.WdError):
        W.wd_set_wait_limit((1 << 26) + 1)
