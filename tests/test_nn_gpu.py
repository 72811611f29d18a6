"""Learned preconditioner on the GPU against the numpy/C oracles.

* the on-device sample generator follows the same counter-based definition
  as the host generator;
* one network layer (tensor-core contraction, BF16 operands, FP32
  accumulation) is within the BF16 rounding bound of the FP64 layer, element
  by element, for every channel shape, on ragged tiles;
* the weight gradient of backpropagation equals its FP64 definition;
* the library's initial weights are the hopping series, and the network then
  reproduces 1 + kH + k^2H^2 + k^3H^3 of the C oracle;
* flexible GCR (plain and preconditioned) reaches 1e-10 on the true residual
  measured by the oracle; training lowers the loss; the preconditioner cuts
  the iteration count.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from oracle import nn
from synth import fields
from tests._wdutil import dev, host, pack_gauge, unpack_spinor
from tests.test_nn_oracle import series_weights

pytestmark = pytest.mark.gpu


def pack_channels(phi, dims):
    """complex [V, C, 3] (lexicographic) -> the documented packed FP32 full
    layout with C channels (blocks of 32 sites, 3C/2 16-byte groups)."""
    V, C = phi.shape[0], phi.shape[1]
    NG = 3 * C // 2
    vh = V // 2
    vh_pad = (vh + 31) // 32 * 32
    half = (vh_pad * C * 24 + 255) // 256 * 256
    buf = np.zeros(2 * half // 4, dtype=np.float32)
    par = fields.site_parity(dims)
    flat = phi.reshape(V, 3 * C)
    for p in (0, 1):
        idx = np.nonzero(par == p)[0]
        cb = idx >> 1
        for k in range(NG):
            off = ((cb >> 5) * NG + k) * 32 + (cb & 31)
            base = p * half // 4 + off * 4
            buf[base + 0] = flat[idx, 2 * k].real
            buf[base + 1] = flat[idx, 2 * k].imag
            buf[base + 2] = flat[idx, 2 * k + 1].real
            buf[base + 3] = flat[idx, 2 * k + 1].imag
    return torch.from_numpy(buf).cuda()


def unpack_channels(t, dims, C):
    V = fields.volume(dims)
    NG = 3 * C // 2
    vh_pad = (V // 2 + 31) // 32 * 32
    half = (vh_pad * C * 24 + 255) // 256 * 256
    buf = t.cpu().numpy().view(np.float32)
    out = np.zeros((V, 3 * C), dtype=np.complex128)
    par = fields.site_parity(dims)
    for p in (0, 1):
        idx = np.nonzero(par == p)[0]
        cb = idx >> 1
        for k in range(NG):
            off = ((cb >> 5) * NG + k) * 32 + (cb & 31)
            base = p * half // 4 + off * 4
            out[idx, 2 * k] = buf[base + 0] + 1j * buf[base + 1]
            out[idx, 2 * k + 1] = buf[base + 2] + 1j * buf[base + 3]
    return out.reshape(V, C, 3)


def test_channel_layout_matches_spinor_packing():
    dims = (4, 4, 4, 8)
    psi = fields.gaussian_spinor(dims)
    a = pack_channels(psi, dims)
    b = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    W.wd_pack_spinor(b, dev(psi), dims, W.WD_FULL, W.WD_F32)
    assert torch.equal(a.view(torch.uint8), b)


def test_device_generator_matches_host_definition():
    dims = (4, 6, 4, 8)
    out = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    W.wd_gaussian_spinor(out, 5678, 2, 0, dims)
    got = unpack_spinor(out, dims, W.WD_FULL, W.WD_F32)
    want = fields.gaussian_spinor(dims, seed=5678)
    assert np.max(np.abs(got - want)) < 2e-6


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("cin,cout", [(4, 8), (8, 8), (8, 4), (4, 4)])
def test_layer_within_bf16_bound(dims, cin, cout):
    U = fields.su3_links(dims, workers=1)
    r = np.random.default_rng(cin * 10 + cout + dims[0])
    Wc = (r.normal(size=(9, cout, cin)) + 1j * r.normal(size=(9, cout, cin))) * 0.3
    phi = r.normal(size=(fields.volume(dims), cin, 3)) + 1j * r.normal(size=(fields.volume(dims), cin, 3))
    g = pack_gauge(U, dims, W.WD_F32, 12)
    out = torch.zeros(W.nn_field_bytes(dims, cout) // 4, dtype=torch.float32, device="cuda")
    w = torch.from_numpy(np.stack([Wc.real, Wc.imag], -1).reshape(-1).astype(np.float32)).cuda()
    W.wd_nn_layer(out, pack_channels(phi, dims), w, cin, cout, g, dims)
    got = unpack_channels(out, dims, cout)
    # the FP64 layer of the FP32-rounded inputs the kernel sees
    phi32 = phi.astype(np.complex64).astype(np.complex128)
    U32 = U.astype(np.complex64).astype(np.complex128)
    want = nn.layer(phi32, U32, Wc.astype(np.complex64).astype(np.complex128), dims)
    # BF16 rounding of both real operands: |err| <= 2 * 2^-8 * sum |W| |T phi|
    tr = nn.transports(dims)
    bound = np.zeros_like(want.real)
    for d in range(9):
        t = np.abs(nn.transport(phi32, U32, dims, d, tr))
        bound += np.einsum("oi,xia->xoa", np.abs(Wc[d]), t)
    err = np.abs(got - want)
    assert np.all(err <= 2 * 2.0 ** -8 * np.sqrt(2) * bound + 1e-5)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 5e-3


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 2, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("cin,cout", [(4, 8), (8, 8), (8, 4)])
def test_weight_gradient(dims, cin, cout):
    """The tensor-core weight gradient (BF16 operands, FP32 accumulation in
    TMEM, fixed-order FP32 sum over CTAs) against its FP64 definition, element
    by element within the BF16 rounding bound, on ragged 32-site blocks."""
    U = fields.su3_links(dims, workers=1)
    r = np.random.default_rng(7 + cin + cout + dims[0])
    V = fields.volume(dims)
    phi = r.normal(size=(V, cin, 3)) + 1j * r.normal(size=(V, cin, 3))
    dl = r.normal(size=(V, cout, 3)) + 1j * r.normal(size=(V, cout, 3))
    g = pack_gauge(U, dims, W.WD_F32, 12)
    grad = torch.zeros(9 * cout * cin * 2, dtype=torch.float32, device="cuda")
    W.wd_nn_wgrad(grad, pack_channels(phi, dims), pack_channels(dl, dims), cin, cout, g, dims)
    got = grad.cpu().numpy().astype(np.float64).reshape(9, cout, cin, 2)
    got = got[..., 0] + 1j * got[..., 1]
    tr = nn.transports(dims)
    ts = [nn.transport(phi, U, dims, d, tr) for d in range(9)]
    want = np.stack([np.einsum("xoa,xia->oi", dl, np.conj(t)) for t in ts])
    # each real product of BF16-rounded operands is off by at most 2 * 2^-8
    # of its size; the FP32 sums add far less
    bound = np.stack([np.einsum("xoa,xia->oi", np.abs(dl), np.abs(t)) for t in ts])
    err = np.abs(got - want)
    assert np.all(err <= 2 * 2.0 ** -8 * 2 * bound + 1e-4)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-2


def test_initial_weights_are_the_hopping_series():
    dims, kappa = (4, 4, 4, 8), 0.13
    w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
    W.wd_nn_init(w, kappa)
    got = nn.split_weights(w.cpu().numpy())
    for a, b in zip(got, series_weights(kappa)):
        assert np.max(np.abs(a - b)) < 1e-7
    # and the network applies 1 + kH + k^2 H^2 + k^3 H^3 (three BF16 layers)
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=43)
    g = pack_gauge(U, dims, W.WD_F32, 12)
    inp = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    W.wd_pack_spinor(inp, dev(b), dims, W.WD_FULL, W.WD_F32)
    out = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    W.wd_nn_apply(out, inp, w, g, dims)
    y = unpack_spinor(out, dims, W.WD_FULL, W.WD_F32)
    want, t = b.copy(), b
    for _ in range(3):
        t = kappa * oracle.hop(t, U, dims)
        want = want + t
    assert np.linalg.norm(y - want) / np.linalg.norm(want) < 2e-2


def solve(dims, kappa, weights=None, m=10, seed=61):
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=seed)
    x = np.zeros_like(b)
    info = W.wd_solve_fgcr(x, b, U, kappa, dims, weights, m)
    r = np.linalg.norm(b - oracle.apply_D(x, U, dims, kappa)) / np.linalg.norm(b)
    return info, r, U


@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.12), ((4, 4, 4, 8), 0.137),
                                        ((6, 6, 6, 6), 0.135)])
def test_gcr_plain_and_preconditioned(dims, kappa):
    info0, r0, _ = solve(dims, kappa)
    assert info0["status"] == W.WD_OK and r0 <= 1.05e-10
    w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
    W.wd_nn_init(w, kappa)
    info1, r1, _ = solve(dims, kappa, w)
    assert info1["status"] == W.WD_OK and r1 <= 1.05e-10
    assert info1["iters"] < info0["iters"]


def test_training_lowers_loss_and_trained_network_preconditions():
    dims, kappa = (4, 4, 4, 8), 0.137
    U = fields.su3_links(dims, workers=1)
    w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
    # start from the identity network (self weights only)
    Ws = [np.zeros((9, 8, 4), complex), np.zeros((9, 8, 8), complex), np.zeros((9, 4, 8), complex)]
    for Wl in Ws:
        for o in range(min(Wl.shape[1], Wl.shape[2])):
            Wl[0, o, o] = 1
    w.copy_(torch.from_numpy(nn.join_weights(Ws)))
    p = W.wd_nn_train_params_default()
    p.init = 0
    p.samples = 512
    p.batch = 8
    p.epochs = 2
    info = W.wd_nn_train(w, U, kappa, dims, p)
    assert info["loss_last"] < 0.8 * info["loss_first"], info
    b = fields.gaussian_spinor(dims, seed=62)
    x = np.zeros_like(b)
    res = W.wd_solve_fgcr(x, b, U, kappa, dims, w, 10)
    r = np.linalg.norm(b - oracle.apply_D(x, U, dims, kappa)) / np.linalg.norm(b)
    assert res["status"] == W.WD_OK and r <= 1.05e-10


def test_training_with_damped_samples():
    """smooth = k damps every other training vector k times with
    x <- x - w D^+ D x before the pair (D x, x) is formed; training still runs
    to finite, decreasing losses and the network still preconditions."""
    dims, kappa = (4, 4, 4, 8), 0.13
    U = fields.su3_links(dims, workers=1)
    # from the identity network (the series start is already near its best)
    Ws = [np.zeros((9, 8, 4), complex), np.zeros((9, 8, 8), complex), np.zeros((9, 4, 8), complex)]
    for Wl in Ws:
        for o in range(min(Wl.shape[1], Wl.shape[2])):
            Wl[0, o, o] = 1
    w = torch.from_numpy(nn.join_weights(Ws)).cuda()
    p = W.wd_nn_train_params_default()
    p.init = 0
    p.samples = 512
    p.batch = 8
    p.epochs = 2
    p.smooth = 4
    info = W.wd_nn_train(w, U, kappa, dims, p)
    assert np.isfinite(info["loss_first"]) and np.isfinite(info["loss_last"])
    assert info["loss_last"] < 0.8 * info["loss_first"], info
    b = fields.gaussian_spinor(dims, seed=63)
    x = np.zeros_like(b)
    res = W.wd_solve_fgcr(x, b, U, kappa, dims, w, 10)
    r = np.linalg.norm(b - oracle.apply_D(x, U, dims, kappa)) / np.linalg.norm(b)
    assert res["status"] == W.WD_OK and r <= 1.05e-10
    p.smooth = -1
    with pytest.raises(W.WdError):
        W.wd_nn_train(w, U, kappa, dims, p)


def _net_case(dims, seed=5):
    """series weights at kappa 0.13 plus random complex weights of size 0.05:
    a well-conditioned network that uses every direction and channel"""
    r = np.random.default_rng(seed)
    Ws = series_weights(0.13)
    Ws = [w + 0.05 * (r.normal(size=w.shape) + 1j * r.normal(size=w.shape)) for w in Ws]
    wdev = torch.from_numpy(nn.join_weights(Ws)).cuda()
    U = fields.su3_links(dims, workers=1)
    b = fields.gaussian_spinor(dims, seed=seed + 1)
    g = pack_gauge(U, dims, W.WD_F32, 12)
    return Ws, wdev, U, b, g


def _apply(flags, wdev, b, g, dims):
    inp = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    W.wd_pack_spinor(inp, dev(b), dims, W.WD_FULL, W.WD_F32)
    out = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    out.zero_()
    if flags is None:
        W.wd_nn_apply(out, inp, wdev, g, dims)
    else:
        W.wd_nn_apply_ex(out, inp, wdev, g, dims, flags)
    return unpack_spinor(out, dims, W.WD_FULL, W.WD_F32)


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 4, 6)])
def test_nn_apply_ex_even_block_and_fp32(dims):
    """flags 0 is wd_nn_apply bit for bit; the even-even block (WD_NN_EVEN)
    equals, bit for bit, the full network applied to the input with its odd
    half set to zero (the directions it skips contribute exact zeros), and
    matches the FP64 network of the oracle within the bound of the FP32
    path."""
    Ws, wdev, U, b, g = _net_case(dims)
    assert np.array_equal(_apply(0, wdev, b, g, dims), _apply(None, wdev, b, g, dims))
    par = fields.site_parity(dims)
    be = b.copy()
    be[par == 1] = 0
    even = _apply(W.WD_NN_EVEN, wdev, b, g, dims)
    full = _apply(0, wdev, be, g, dims)
    assert np.array_equal(even[par == 0], full[par == 0])
    want = nn.network(be, U, Ws, dims)[par == 0]
    assert np.linalg.norm(even[par == 0] - want) / np.linalg.norm(want) < 2e-2


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 4, 6)])
@pytest.mark.parametrize("even", [False, True])
def test_nn_apply_ex_bf16_activations(dims, even):
    """BF16 activations (WD_NN_BF16), alone and with the even-even block,
    against the FP64 network of the oracle.  Per layer the operands of the
    link transport (activations, link entries) are rounded to BF16 (8
    significant bits, 2^-9 relative) and each packed multiply-add rounds to
    BF16 again; with the BF16 tensor-core operands of the FP32 path this adds
    a few 2^-9 per layer, so three layers stay below 3e-2 relative (measured
    about 1e-2)."""
    Ws, wdev, U, b, g = _net_case(dims, seed=7)
    par = fields.site_parity(dims)
    src = b.copy()
    if even:
        src[par == 1] = 0
    got = _apply(W.WD_NN_BF16 | (W.WD_NN_EVEN if even else 0), wdev, b if not even else b, g,
                 dims)
    want = nn.network(src, U, Ws, dims)
    sel = (par == 0) if even else np.ones(len(par), bool)
    err = np.linalg.norm(got[sel] - want[sel]) / np.linalg.norm(want[sel])
    assert err < 3e-2, err


@pytest.mark.parametrize("even", [False, True])
def test_nn_apply_ex_bf16_one_thread_per_site_kernel(even):
    """On 16^3x64 the BF16 layers with at least two waves of tiles run the
    one-thread-per-site inference kernel (the full-lattice layers here; the
    even-only last layer of the even block, with half the tiles, runs the
    two-thread kernel): the same bound against the FP64 network."""
    dims = (16, 16, 16, 64)
    Ws, wdev, U, b, g = _net_case(dims, seed=7)
    par = fields.site_parity(dims)
    src = b.copy()
    if even:
        src[par == 1] = 0
    got = _apply(W.WD_NN_BF16 | (W.WD_NN_EVEN if even else 0), wdev, b, g, dims)
    want = nn.network(src, U, Ws, dims)
    sel = (par == 0) if even else np.ones(len(par), bool)
    err = np.linalg.norm(got[sel] - want[sel]) / np.linalg.norm(want[sel])
    assert err < 3e-2, err


def test_nn_apply_ex_rejects_unknown_flags():
    dims = (4, 4, 4, 4)
    _, wdev, _, b, g = _net_case(dims)
    inp = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    out = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
    with pytest.raises(W.WdError):
        W.wd_nn_apply_ex(out, inp, wdev, g, dims, 4)
