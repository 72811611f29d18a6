"""Helpers for the GPU tests: move canonical numpy fields through libwd's
pack/unpack entry points (argument marshalling only)."""
import numpy as np
import torch

import paper_0810_5365_gb300 as W

PREC_TOL = {W.WD_F64: 1e-13, W.WD_F32: 1e-6, W.WD_F16: 5e-3}
PREC_NAME = {W.WD_F64: "f64", W.WD_F32: "f32", W.WD_F16: "f16"}

# Relative bound on a reported norm or dot product against numpy's FP64 sum of
# the stored values.  Each site's 24 terms are summed in the working precision
# (FP32 for the FP32/FP16 fields): 24 positive terms in float carry at most
# 24 * 2^-24 = 1.4e-6 relative error; the sum over sites is FP64.
NORM_TOL = {W.WD_F64: 1e-12, W.WD_F32: 2e-6, W.WD_F16: 2e-6}


def dev(a):
    """complex128 numpy array -> contiguous float64 CUDA tensor (same bytes)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).copy()).cuda()


def host(t, shape):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def pack_spinor(psi, dims, parity, prec):
    buf = W.alloc_spinor(dims, parity, prec)
    src = dev(psi)
    W.wd_pack_spinor(buf, src, dims, parity, prec)
    torch.cuda.synchronize()
    return buf


def unpack_spinor(buf, dims, parity, prec):
    V = int(np.prod(dims))
    n = V if parity == W.WD_FULL else V // 2
    out = torch.empty(n * 24, dtype=torch.float64, device="cuda")
    W.wd_unpack_spinor(out, buf, dims, parity, prec)
    return host(out, (n, 4, 3))


def pack_gauge(U, dims, prec, recon):
    buf = W.alloc_gauge(dims, prec, recon)
    W.wd_pack_gauge(buf, dev(U), dims, prec, recon)
    torch.cuda.synchronize()
    return buf


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    """largest elementwise error relative to the largest reference magnitude"""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def temporal_gauge_links(U, dims):
    """Links in temporal gauge, made on the host from the definition:
    omega(x, 0) = 1, omega(x, t+1) = omega(x, t) U_t(x, t) and
    U'_mu(x) = omega(x) U_mu(x) omega(x+mu)^+, with U'_t set to the exact
    identity off the last time slice (the form the hopping kernels assume
    under WD_TEMPORAL_GAUGE).  Returns (U', omega)."""
    from tests.test_oracle_pins import gauge_rotate
    V = int(np.prod(dims))
    S = int(dims[0]) * int(dims[1]) * int(dims[2])
    om = np.zeros((V, 3, 3), dtype=np.complex128)
    om[:S] = np.eye(3)
    for t in range(int(dims[3]) - 1):
        om[(t + 1) * S:(t + 2) * S] = om[t * S:(t + 1) * S] @ U[3][t * S:(t + 1) * S]
    Up = gauge_rotate(U, om, dims)
    Up[3][: (int(dims[3]) - 1) * S] = np.eye(3)
    return Up, om
