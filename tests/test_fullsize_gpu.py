"""Parity at the benchmark's full sizes, in the launch configurations
bench.py times, on outputs the oracle computes site by site.

* the 32^3x64 parity dslash (FP32 and FP16 with 12-real links, FP64 with
  18), launched exactly as the headline: wd_dslash_ex, even output, a = -kappa;
  checked on random even sites plus every boundary case (t = 0 and t = L3-1,
  where the antiperiodic sign enters, and the x, y, z wrap faces);
* the mixed-precision solve on 24^3x48 (FP16 inner CG at kappa = 0.137,
  FP16 inner BiCGstab in temporal gauge at kappa = 0.130), judged by the
  oracle's own true residual over the whole lattice;
* the 12-right-hand-side multi-RHS dslash on 24^3x48, sampled per RHS;
* the FP16 kernel with staged z and t neighbours on 32^3x64, bit for bit
  against the unstaged FP16 kernel (both parities, H and H^+), which covers
  the z and t wrap blocks at full size.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import PREC_TOL, pack_gauge, pack_spinor, rel_l2, rel_max, unpack_spinor

pytestmark = pytest.mark.gpu

HEADLINE = (32, 32, 32, 64)
KAPPA = 0.1365
SOLVE = (24, 24, 24, 48)


def _even_samples(dims, n, seed):
    """random even lexicographic sites plus the boundary faces"""
    x = fields.coords(dims)
    par = fields.site_parity(dims)
    r = np.random.default_rng(seed)
    even = np.nonzero(par == 0)[0]
    pick = set(r.choice(even, size=n, replace=False).tolist())
    for mu in range(4):
        for edge in (0, dims[mu] - 1):
            face = np.nonzero((x[:, mu] == edge) & (par == 0))[0]
            pick.update(r.choice(face, size=min(64, len(face)), replace=False).tolist())
    return np.array(sorted(pick), dtype=np.int64)


@pytest.fixture(scope="module")
def headline_fields():
    return fields.su3_links(HEADLINE), fields.gaussian_spinor(HEADLINE)


@pytest.mark.parametrize("dagger", [0, 1])
def test_headline_staged_f16_bit_exact(headline_fields, dagger):
    U, psi = headline_fields
    g = pack_gauge(U, HEADLINE, W.WD_F16, 12)
    for p in (W.WD_EVEN, W.WD_ODD):
        a = pack_spinor(fields.to_half(psi, HEADLINE, 1 - p), HEADLINE, 1 - p, W.WD_F16)
        ref = W.alloc_spinor(HEADLINE, p, W.WD_F16)
        out = W.alloc_spinor(HEADLINE, p, W.WD_F16)
        W.wd_dslash_ex(ref, a, g, p, dagger, -KAPPA, None, 0.0, None, 0.0, None, HEADLINE,
                       W.WD_F16, 12)
        W.wd_dslash_ex(out, a, g, p, dagger, -KAPPA, None, 0.0, None, 0.0, None, HEADLINE,
                       W.WD_F16, 12 | W.WD_STAGE_NEIGHBOURS)
        torch.cuda.synchronize()
        assert W.wd_async_status() == W.WD_OK
        assert torch.equal(out, ref), (p, dagger)


@pytest.mark.parametrize("prec,recon", [(W.WD_F32, 12), (W.WD_F16, 12), (W.WD_F64, 18)])
def test_headline_dslash_sampled(headline_fields, prec, recon):
    U, psi = headline_fields
    g = pack_gauge(U, HEADLINE, prec, recon)
    a = pack_spinor(fields.to_half(psi, HEADLINE, 1), HEADLINE, W.WD_ODD, prec)
    b = W.alloc_spinor(HEADLINE, W.WD_EVEN, prec)
    W.wd_dslash_ex(b, a, g, W.WD_EVEN, 0, -KAPPA, None, 0.0, None, 0.0, None, HEADLINE, prec,
                   recon)
    got = unpack_spinor(b, HEADLINE, W.WD_EVEN, prec)
    sites = _even_samples(HEADLINE, 4096, 11)
    want = -KAPPA * oracle.hop_sites(psi, U, HEADLINE, sites)
    got_s = got[sites >> 1]
    tol = PREC_TOL[prec]
    assert rel_l2(got_s, want) <= tol, rel_l2(got_s, want)
    assert rel_max(got_s, want) <= 4 * tol, rel_max(got_s, want)
    # the time-boundary sites on their own (the antiperiodic sign)
    tb = np.isin(fields.coords(HEADLINE)[sites, 3], (0, HEADLINE[3] - 1))
    assert tb.sum() >= 64
    assert rel_l2(got_s[tb], want[tb]) <= tol


@pytest.fixture(scope="module")
def solve_fields():
    return fields.su3_links(SOLVE), fields.gaussian_spinor(SOLVE, seed=2025)


@pytest.mark.parametrize("kappa,solver,gf", [(0.137, 0, 0), (0.130, 1, 1)])
def test_solve_24x24x24x48_true_residual(solve_fields, kappa, solver, gf):
    U, b = solve_fields
    x = np.zeros_like(b)
    p = W.wd_solve_params_default()
    p.inner_prec = W.WD_F16
    p.solver = solver
    p.gauge_fix = gf
    info = W.wd_solve_ex(x, b, U, kappa, SOLVE, p)
    assert info["status"] == W.WD_OK
    r = np.linalg.norm(b - oracle.apply_D(x, U, SOLVE, kappa)) / np.linalg.norm(b)
    assert r <= 1.05e-10, r


def test_mrhs_12_rhs_24x24x24x48_sampled(solve_fields):
    U, _ = solve_fields
    nr, prec = 12, W.WD_F32
    g = pack_gauge(U, SOLVE, prec, 12)
    h = W.wd_spinor_bytes(SOLVE, W.WD_ODD, prec)
    inp = torch.empty(nr * h, dtype=torch.uint8, device="cuda")
    psis = [fields.gaussian_spinor(SOLVE, seed=900 + r) for r in range(nr)]
    for r in range(nr):
        inp[r * h:(r + 1) * h] = pack_spinor(fields.to_half(psis[r], SOLVE, 1), SOLVE,
                                             W.WD_ODD, prec)
    out = torch.empty_like(inp)
    W.wd_dslash_mrhs(out, inp, g, W.WD_EVEN, 0, -0.136, None, 0.0, nr, None, SOLVE, prec, 12)
    sites = _even_samples(SOLVE, 1024, 12)
    for r in (0, 5, 11):
        got = unpack_spinor(out[r * h:(r + 1) * h], SOLVE, W.WD_EVEN, prec)[sites >> 1]
        want = -0.136 * oracle.hop_sites(psis[r], U, SOLVE, sites)
        assert rel_l2(got, want) <= PREC_TOL[prec]
        assert rel_max(got, want) <= 4 * PREC_TOL[prec]
