"""wd_dslash_ex_noalloc: the allocation-free variant of wd_dslash_ex.

It exists for callers that cannot let libwd call cudaMalloc: code that
records launches into a CUDA graph by stream capture, applications whose
device memory belongs to another allocator, and latency-critical loops that
must not hit the device-wide synchronisation of cudaMalloc/cudaFree.  Its
reduction scratch is a fixed array inside the library, shared by every call.

The GPU test calls it through the C ABI twice in a row (the second call finds
the array as the first left it) and compares the output field and the FP64
norm with wd_dslash_ex's, at the tolerances the parity tests use.  This file
is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import PREC_TOL, pack_gauge, pack_spinor, rel_l2, rel_max, unpack_spinor


def test_noalloc_rejects_lattices_beyond_its_scratch():
    # V/2 = 4,194,304 sites > 2,097,152: refused on the host, nothing queued
    W.wd.lib()
    with pytest.raises(W.WdError) as e:
        W.wd_dslash_ex_noalloc(16, 32, 48, 0, 0, 1.0, None, 0.0, None, 0.0, 64,
                               (64, 64, 64, 32), W.WD_F32, 12)
    assert e.value.status == W.WD_ERR_SCRATCH
    assert "noalloc" in W.wd_error_string(W.WD_ERR_SCRATCH)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F16, 12)])
def test_noalloc_matches_wd_dslash_ex_on_two_calls(prec, recon):
    kappa = 0.1365
    for dims in [(8, 8, 8, 16), (6, 6, 6, 6)]:  # 32 CTAs, then a ragged 6 CTAs
        U = fields.su3_links(dims, workers=1)
        psi = fields.gaussian_spinor(dims)
        odd = fields.to_half(psi, dims, 1)
        ev = fields.to_half(fields.gaussian_spinor(dims, seed=31), dims, 0)
        g = pack_gauge(U, dims, prec, recon)
        inp = pack_spinor(odd, dims, W.WD_ODD, prec)
        x = pack_spinor(ev, dims, W.WD_EVEN, prec)

        ref = W.alloc_spinor(dims, W.WD_EVEN, prec)
        nref = torch.zeros(1, dtype=torch.float64, device="cuda")
        W.wd_dslash_ex(ref, inp, g, W.WD_EVEN, 0, -kappa * kappa, x, 1.0, None, 0.0, nref,
                       dims, prec, recon)
        want = unpack_spinor(ref, dims, W.WD_EVEN, prec)
        for call in range(2):
            out = W.alloc_spinor(dims, W.WD_EVEN, prec)
            n = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            W.wd_dslash_ex_noalloc(out, inp, g, W.WD_EVEN, 0, -kappa * kappa, x, 1.0, None, 0.0,
                                   n, dims, prec, recon)
            got = unpack_spinor(out, dims, W.WD_EVEN, prec)
            tol = PREC_TOL[prec]
            assert rel_l2(got, want) <= tol, (call, rel_l2(got, want))
            assert rel_max(got, want) <= 4 * tol, (call, rel_max(got, want))
            assert abs(n.item() - nref.item()) <= 1e-12 * nref.item(), (call, n.item(), nref.item())


@pytest.mark.gpu
@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F16, 12)])
def test_noalloc_temporal_gauge_links(prec, recon):
    """recon | WD_TEMPORAL_GAUGE, as wd_dslash_ex takes it: the same field and
    norm as wd_dslash_ex, and the oracle's hop on the temporal-gauge links
    (made on the host from their definition), on two calls in a row."""
    from tests._wdutil import temporal_gauge_links
    import oracle

    dims = (6, 4, 4, 8)
    U = fields.su3_links(dims, workers=1)
    Up, _ = temporal_gauge_links(U, dims)
    psi = fields.gaussian_spinor(dims)
    g = pack_gauge(Up, dims, prec, recon)
    flags = recon | W.WD_TEMPORAL_GAUGE
    for p in (W.WD_EVEN, W.WD_ODD):
        src = fields.to_half(psi, dims, 1 - p)
        inp = pack_spinor(src, dims, 1 - p, prec)
        ref = W.alloc_spinor(dims, p, prec)
        nref = torch.zeros(1, dtype=torch.float64, device="cuda")
        W.wd_dslash_ex(ref, inp, g, p, 1, 1.0, None, 0.0, None, 0.0, nref, dims, prec, flags)
        want = oracle.hop_block(p, src, Up, dims, dagger=True)
        for call in range(2):
            out = W.alloc_spinor(dims, p, prec)
            n = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            W.wd_dslash_ex_noalloc(out, inp, g, p, 1, 1.0, None, 0.0, None, 0.0, n, dims, prec,
                                   flags)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (p, call)
            assert n.item() == nref.item(), (p, call)
            got = unpack_spinor(out, dims, p, prec)
            assert rel_l2(got, want) <= PREC_TOL[prec], (p, call)
            assert rel_max(got, want) <= 4 * PREC_TOL[prec], (p, call)


@pytest.mark.gpu
def test_noalloc_staged_neighbours():
    """12 | WD_STAGE_NEIGHBOURS through the allocation-free entry point: bit
    for bit the unstaged FP16 field, with no fault raised; and the flag
    combinations that wd_dslash_ex refuses are refused here too."""
    dims = (8, 8, 6, 4)
    U = fields.su3_links(dims, workers=1)
    g = pack_gauge(U, dims, W.WD_F16, 12)
    inp = pack_spinor(fields.to_half(fields.gaussian_spinor(dims), dims, 1), dims, 1, W.WD_F16)
    ref = W.alloc_spinor(dims, 0, W.WD_F16)
    W.wd_dslash_ex(ref, inp, g, 0, 0, -0.13, None, 0.0, None, 0.0, None, dims, W.WD_F16, 12)
    for call in range(2):
        out = W.alloc_spinor(dims, 0, W.WD_F16)
        W.wd_dslash_ex_noalloc(out, inp, g, 0, 0, -0.13, None, 0.0, None, 0.0, None, dims,
                               W.WD_F16, 12 | W.WD_STAGE_NEIGHBOURS)
        assert W.wd_async_status() == W.WD_OK
        assert torch.equal(out, ref), call
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    for recon, norm in [(12 | W.WD_STAGE_NEIGHBOURS, nrm),
                        (12 | W.WD_STAGE_NEIGHBOURS | W.WD_TEMPORAL_GAUGE, None)]:
        with pytest.raises(W.WdError) as e:
            W.wd_dslash_ex_noalloc(out, inp, g, 0, 0, 1.0, None, 0.0, None, 0.0, norm, dims,
                                   W.WD_F16, recon)
        assert e.value.status == W.WD_ERR_ARG
