"""Multi-right-hand-side hopping kernel and batched solves (GPU), against the
FP64 oracle.

The multi-RHS kernel is checked right-hand side by right-hand side with the
parity tolerances of the single-field kernel.  The batched solver is judged
by the oracle's own true residual on every unpacked solution, on a batch
that mixes lattice sizes (ragged tiles) and point sources, and on its
per-right-hand-side masking (right-hand sides that converge early stop
while the others go on).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0810_5365_gb300 as W
from synth import fields
from tests._wdutil import NORM_TOL, PREC_TOL, dev, pack_gauge, rel_l2, rel_max, unpack_spinor

pytestmark = pytest.mark.gpu


def pack_many(fs, dims, parity, prec):
    h = W.wd_spinor_bytes(dims, parity, prec)
    buf = torch.empty(h * len(fs), dtype=torch.uint8, device="cuda")
    for r, f in enumerate(fs):
        W.wd_pack_spinor(buf[r * h:(r + 1) * h], dev(f), dims, parity, prec)
    return buf, h


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 6, 6, 6), (2, 4, 2, 6)])
@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F32, 18),
                                        (W.WD_F16, 12)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_mrhs_dslash_matches_oracle(dims, prec, recon, dagger):
    nrhs = 5
    U = fields.su3_links(dims, workers=1)
    g = pack_gauge(U, dims, prec, recon)
    srcs = [oracle.restrict(fields.gaussian_spinor(dims, seed=100 + r), dims, 1)
            for r in range(nrhs)]
    xs = [oracle.restrict(fields.gaussian_spinor(dims, seed=200 + r), dims, 0)
          for r in range(nrhs)]
    inp, h = pack_many(srcs, dims, 1, prec)
    out, _ = pack_many(xs, dims, 0, prec)  # x aliases out
    nrm = torch.zeros(nrhs, dtype=torch.float64, device="cuda")
    a, bx = -0.137 ** 2, 1.0
    W.wd_dslash_mrhs(out, inp, g, 0, dagger, a, out, bx, nrhs, nrm, dims, prec, recon)
    torch.cuda.synchronize()
    for r in range(nrhs):
        got = unpack_spinor(out[r * h:(r + 1) * h], dims, 0, prec)
        want = a * oracle.hop_block(0, srcs[r], U, dims, dagger=bool(dagger)) + bx * xs[r]
        tol = PREC_TOL[prec]
        assert rel_l2(got, want) <= tol, (r, rel_l2(got, want))
        assert rel_max(got, want) <= 4 * tol
        n2 = np.vdot(got, got).real
        assert abs(nrm[r].item() - n2) <= NORM_TOL[prec] * n2


def _mrhs_run(dims, prec, recon, nrhs, dagger=0):
    U = fields.su3_links(dims, workers=1)
    g = pack_gauge(U, dims, prec, recon)
    srcs = [oracle.restrict(fields.gaussian_spinor(dims, seed=700 + r), dims, 1)
            for r in range(nrhs)]
    xs = [oracle.restrict(fields.gaussian_spinor(dims, seed=800 + r), dims, 0)
          for r in range(nrhs)]
    inp, h = pack_many(srcs, dims, 1, prec)
    out, _ = pack_many(xs, dims, 0, prec)
    nrm = torch.zeros(nrhs, dtype=torch.float64, device="cuda")
    W.wd_dslash_mrhs(out, inp, g, 0, dagger, -0.13, out, 1.0, nrhs, nrm, dims, prec, recon)
    torch.cuda.synchronize()
    return out, nrm, h, U, srcs, xs


PAIR = 16  # shape code: two right-hand sides per thread (FP32)


@pytest.mark.parametrize("lanes", [1, 2, 8, PAIR + 1, PAIR + 2, PAIR + 4])
@pytest.mark.parametrize("prec,recon", [(W.WD_F64, 18), (W.WD_F32, 12), (W.WD_F32, 18),
                                        (W.WD_F16, 12)])
def test_mrhs_every_tile_shape(lanes, prec, recon):
    """Every tile shape the autotuner may choose gives bit-identical fields and
    norms to the default shape (every right-hand side of every site goes
    through the same operations in the same order, whether a thread holds one
    right-hand side or two), and both match the oracle; 6x4x4x6 has a ragged
    last tile and nrhs = 7 leaves idle lanes for lanes = 2, 8 and a thread
    whose second right-hand side does not exist for the pair shapes (FP64 and
    FP16 run the pair codes as the one-per-thread shape with as many warps)."""
    dims, nrhs = (6, 4, 4, 6), 7
    try:
        W.wd_mrhs_set_lanes(4)
        ref, nref, h, U, srcs, xs = _mrhs_run(dims, prec, recon, nrhs, dagger=1)
        W.wd_mrhs_set_lanes(lanes)
        got, ngot, _, _, _, _ = _mrhs_run(dims, prec, recon, nrhs, dagger=1)
    finally:
        W.wd_mrhs_set_lanes(0)
    # compare the stored sites (the FP16 half field has pad bytes after its
    # scales that no kernel writes)
    assert torch.equal(nref, ngot)
    for r in range(nrhs):
        g = unpack_spinor(got[r * h:(r + 1) * h], dims, 0, prec)
        assert np.array_equal(g, unpack_spinor(ref[r * h:(r + 1) * h], dims, 0, prec))
        want = -0.13 * oracle.hop_block(0, srcs[r], U, dims, dagger=True) + xs[r]
        assert rel_l2(g, want) <= PREC_TOL[prec]


def test_mrhs_set_lanes_rejects_other_shapes():
    for bad in (3, PAIR, PAIR + 8):
        with pytest.raises(W.WdError):
            W.wd_mrhs_set_lanes(bad)


def test_batched_solve_pair_shape_is_bit_identical():
    """A batched solve whose hopping launches hold two right-hand sides per
    thread gives the same solutions, bit for bit, and the same iteration
    counts as one right-hand side per thread.  The batch's right-hand sides
    converge at different iterations, so the convergence mask switches off
    one member of a thread's pair while the other goes on.  (Tile shapes
    belong to the per-step launches: batch mode 0.)"""
    prev = W.wd_set_batch_mode(0)
    try:
        W.wd_mrhs_set_lanes(2)
        rc1, i1, k1 = _batch(W.WD_F32)
        W.wd_mrhs_set_lanes(PAIR + 2)
        rc2, i2, k2 = _batch(W.WD_F32)
    finally:
        W.wd_mrhs_set_lanes(0)
        W.wd_set_batch_mode(prev)
    assert rc1 == rc2 == W.WD_OK
    assert len({d["iters"] for d in i1}) > 1
    assert [d["iters"] for d in i1] == [d["iters"] for d in i2]
    for (_, _, _, x1), (_, _, _, x2) in zip(k1, k2):
        assert np.array_equal(x1, x2)


def test_autotuner_times_every_shape_and_leaves_outputs_alone():
    """A new FP32 batch shape is timed with all seven tile shapes on temporary
    outputs: the caller's output equals the untuned (default-shape) result
    exactly, and the report lists the shape with seven timings and a choice."""
    dims, prec, nrhs = (8, 4, 6, 10), W.WD_F32, 6
    prev = W.wd_set_autotune(0)
    try:
        W.wd_mrhs_set_lanes(4)
        ref, nref, h, _, _, _ = _mrhs_run(dims, prec, 12, nrhs)
        W.wd_mrhs_set_lanes(0)
        W.wd_set_autotune(1)
        got, ngot, _, _, _, _ = _mrhs_run(dims, prec, 12, nrhs)
    finally:
        W.wd_mrhs_set_lanes(0)
        W.wd_set_autotune(prev)
    assert torch.equal(nref, ngot)
    for r in range(nrhs):
        assert np.array_equal(unpack_spinor(got[r * h:(r + 1) * h], dims, 0, prec),
                              unpack_spinor(ref[r * h:(r + 1) * h], dims, 0, prec))
    n, text = W.wd_tune_report()
    assert n >= 1
    tiles = (int(np.prod(dims)) // 2 + 127) // 128
    mine = [l for l in text.splitlines()
            if f"tiles={tiles} " in l and f"maxrhs={nrhs} " in l and "norm=1" in l]
    assert len(mine) == 1, text
    us = [float(v) for v in mine[0].split("us[1,2,4,8,p1,p2,p4]=")[1].split()[0].split(",")]
    assert len(us) == 7 and all(v > 0 for v in us)
    shape = mine[0].split("shape=")[1].strip()
    names = ["1", "2", "4", "8", "p1", "p2", "p4"]
    assert shape in names and us[names.index(shape)] == min(us)


def test_mrhs_agrees_with_single_rhs_kernel():
    """The multi-RHS kernel and the single-field kernel agree to FP32 rounding."""
    dims, prec = (8, 8, 8, 8), W.WD_F32
    U = fields.su3_links(dims, workers=1)
    g = pack_gauge(U, dims, prec, 12)
    srcs = [oracle.restrict(fields.gaussian_spinor(dims, seed=300 + r), dims, 0) for r in range(3)]
    inp, h = pack_many(srcs, dims, 0, prec)
    out = torch.empty_like(inp)
    W.wd_dslash_mrhs(out, inp, g, 1, 0, -0.1365, None, 0.0, 3, None, dims, prec, 12)
    for r in range(3):
        one = W.alloc_spinor(dims, 1, prec)
        W.wd_dslash(one, inp[r * h:(r + 1) * h], g, 0.1365, 1, dims, prec)
        a = unpack_spinor(one, dims, 1, prec)
        b = unpack_spinor(out[r * h:(r + 1) * h], dims, 1, prec)
        assert rel_l2(a, b) <= 1e-6


def _batch(prec, use_graph=1):
    """Mixed lattices with Gaussian right-hand sides plus point sources."""
    probs, keep = [], []
    spec = [((4, 4, 4, 4), 3, "gauss"), ((6, 6, 6, 6), 2, "gauss"), ((4, 4, 4, 8), 4, "point")]
    for j, (dims, nrhs, kind) in enumerate(spec):
        U = fields.su3_links(dims, seed=1234 + j, workers=1)
        if kind == "gauss":
            bs = [fields.gaussian_spinor(dims, seed=500 + 10 * j + r) for r in range(nrhs)]
        else:
            bs = [fields.point_source(dims, 0, r % 4, r % 3) for r in range(nrhs)]
        b = np.ascontiguousarray(np.stack(bs))
        x = np.zeros_like(b)
        probs.append({"dims": dims, "kappa": 0.136, "nrhs": nrhs, "gauge": U, "b": b, "x": x})
        keep.append((dims, U, b, x))
    p = W.wd_solve_params_default()
    p.inner_prec = prec
    p.use_graph = use_graph
    rc, infos = W.wd_solve_batch(probs, p)
    return rc, infos, keep


@pytest.mark.parametrize("prec", [W.WD_F32, W.WD_F16, W.WD_F64])
def test_batched_solve_true_residuals(prec):
    rc, infos, keep = _batch(prec)
    assert rc == W.WD_OK
    k = 0
    for dims, U, b, x in keep:
        for r in range(b.shape[0]):
            res = b[r] - oracle.apply_D(x[r], U, dims, 0.136)
            rel = np.linalg.norm(res) / np.linalg.norm(b[r])
            assert rel <= 1.05e-10, (dims, r, rel)
            assert infos[k]["status"] == W.WD_OK and infos[k]["true_residual"] <= 1e-10
            k += 1


def test_batched_matches_single_solves_iteration_counts():
    """Each right-hand side of a batch follows the same recurrence as a
    single solve: its iteration count matches wd_solve_ex's."""
    rc, infos, keep = _batch(W.WD_F32)
    dims, U, b, _ = keep[0]
    for r in range(b.shape[0]):
        x = np.zeros_like(b[r])
        one = W.wd_solve_ex(x, b[r], U, 0.136, dims)
        assert abs(one["iters"] - infos[r]["iters"]) <= 10


@pytest.mark.parametrize("mode", [1, 0])
def test_batched_graph_and_plain_agree(mode):
    """Captured graph and direct launches give the same iterates bit for bit,
    in both batch modes (one persistent launch per iteration, one launch per
    step)."""
    prev = W.wd_set_batch_mode(mode)
    try:
        rc1, i1, k1 = _batch(W.WD_F32, use_graph=1)
        rc2, i2, k2 = _batch(W.WD_F32, use_graph=0)
    finally:
        W.wd_set_batch_mode(prev)
    assert rc1 == rc2 == W.WD_OK
    for (_, _, _, x1), (_, _, _, x2) in zip(k1, k2):
        assert np.array_equal(x1, x2)
    assert [d["iters"] for d in i1] == [d["iters"] for d in i2]


@pytest.mark.parametrize("prec", [W.WD_F32, W.WD_F16])
def test_persistent_iteration_matches_per_step_launches(prec):
    """One persistent cooperative launch per iteration against one launch per
    step: the same algorithm up to the summation order of the norms, so every
    right-hand side converges (oracle residual) in the same number of
    iterations to within one check interval, and two persistent runs agree
    bit for bit (fixed-order reductions)."""
    out = {}
    prev = W.wd_set_batch_mode(1)
    try:
        for mode in (1, 0, 1):
            W.wd_set_batch_mode(mode)
            rc, infos, keep = _batch(prec)
            assert rc == W.WD_OK, mode
            for dims, U, b, x in keep:
                for r in range(b.shape[0]):
                    rel = (np.linalg.norm(b[r] - oracle.apply_D(x[r], U, dims, 0.136))
                           / np.linalg.norm(b[r]))
                    assert rel <= 1.05e-10, (mode, dims, r, rel)
            out.setdefault(mode, []).append((infos, [k[3].copy() for k in keep]))
    finally:
        W.wd_set_batch_mode(prev)
    (i1, x1), (i1b, x1b) = out[1]
    (i0, _), = out[0]
    for a, b in zip(x1, x1b):
        assert np.array_equal(a, b)
    assert [d["iters"] for d in i1] == [d["iters"] for d in i1b]
    for a, b in zip(i1, i0):
        assert abs(a["iters"] - b["iters"]) <= 10, (a["iters"], b["iters"])


def test_persistent_iteration_barrier_timeout():
    """The failure path of the grid barriers, run on purpose and without any
    fault: with a wait limit of 0 polls every CTA but the last to arrive gives
    up at the first barrier, raises the error word and leaves, the others see
    it at their next barrier and leave, and the solve returns WD_ERR_TIMEOUT.
    The next solve with the default limit is exact."""
    prev = W.wd_set_batch_mode(1)
    try:
        W.wd_set_wait_limit(0)
        dims = (4, 4, 4, 8)
        U = fields.su3_links(dims, workers=1)
        b = np.ascontiguousarray(np.stack([fields.gaussian_spinor(dims, seed=s)
                                           for s in (11, 12, 13)]))
        x = np.zeros_like(b)
        pr = [{"dims": dims, "kappa": 0.13, "nrhs": 3, "gauge": U, "b": b, "x": x}]
        rc, _ = W.wd_solve_batch(pr, check=False)
        assert rc == W.WD_ERR_TIMEOUT
    finally:
        W.wd_set_wait_limit(1 << 22)
        W.wd_set_batch_mode(prev)
    x[:] = 0
    rc, infos = W.wd_solve_batch(pr)
    assert rc == W.WD_OK
    for r in range(3):
        rel = np.linalg.norm(b[r] - oracle.apply_D(x[r], U, dims, 0.13)) / np.linalg.norm(b[r])
        assert rel <= 1.05e-10


def test_batch_mode_rejects_other_values():
    with pytest.raises(W.WdError):
        W.wd_set_batch_mode(2)


def test_batch_device_buffers():
    dims = (4, 4, 4, 8)
    U = fields.su3_links(dims, workers=1)
    b = np.ascontiguousarray(np.stack([fields.gaussian_spinor(dims, seed=s) for s in (1, 2)]))
    bd, Ud = dev(b), dev(U)
    xd = torch.zeros_like(bd)
    rc, infos = W.wd_solve_batch([{"dims": dims, "kappa": 0.13, "nrhs": 2, "gauge": Ud,
                                   "b": bd, "x": xd}])
    x = xd.cpu().numpy().view(np.complex128).reshape(b.shape)
    for r in range(2):
        rel = np.linalg.norm(b[r] - oracle.apply_D(x[r], U, dims, 0.13)) / np.linalg.norm(b[r])
        assert rel <= 1.05e-10


def test_batch_at_its_limits():
    """16 problems (the most a batch takes) of assorted shapes, one of them
    with 32 right-hand sides (the most a problem takes): every solution meets
    the oracle's true residual."""
    r = np.random.default_rng(17)
    shapes = [(4, 4, 4, 4), (2, 4, 2, 6), (6, 4, 4, 6), (4, 2, 4, 8), (2, 2, 2, 2),
              (4, 6, 2, 4), (8, 4, 2, 4), (2, 6, 4, 4)]
    probs, keep = [], []
    for j in range(16):
        dims = shapes[j % len(shapes)]
        nrhs = 32 if j == 5 else int(r.integers(1, 4))
        U = fields.su3_links(dims, seed=3000 + j, workers=1)
        b = np.ascontiguousarray(np.stack([fields.gaussian_spinor(dims, seed=4000 + 40 * j + k)
                                           for k in range(nrhs)]))
        x = np.zeros_like(b)
        probs.append({"dims": dims, "kappa": 0.125, "nrhs": nrhs, "gauge": U, "b": b, "x": x})
        keep.append((dims, U, b, x))
    p = W.wd_solve_params_default()
    rc, infos = W.wd_solve_batch(probs, p)
    assert rc == W.WD_OK and len(infos) == sum(pr["nrhs"] for pr in probs)
    for dims, U, b, x in keep:
        for k in range(b.shape[0]):
            res = b[k] - oracle.apply_D(x[k], U, dims, 0.125)
            assert np.linalg.norm(res) / np.linalg.norm(b[k]) <= 1.05e-10


def test_batched_resume_from_initial_guess():
    """A batched solve restarted from the partial solutions of a loose first
    pass (nonzero x: the FP64 residual is formed in setup) reaches 1e-10 on
    every right-hand side in fewer iterations than a start from zero."""
    probs, keep = [], []
    for j, (dims, nrhs) in enumerate([((4, 4, 4, 4), 2), ((6, 4, 4, 6), 3)]):
        U = fields.su3_links(dims, seed=5000 + j, workers=1)
        b = np.ascontiguousarray(np.stack([fields.gaussian_spinor(dims, seed=6000 + 10 * j + k)
                                           for k in range(nrhs)]))
        x = np.zeros_like(b)
        probs.append({"dims": dims, "kappa": 0.13, "nrhs": nrhs, "gauge": U, "b": b, "x": x})
        keep.append((dims, U, b, x))
    p = W.wd_solve_params_default()
    p.tol = 1e-5
    rc, loose = W.wd_solve_batch(probs, p)
    assert rc == W.WD_OK
    p.tol = 1e-10
    p.use_initial_guess = 1
    rc, resumed = W.wd_solve_batch(probs, p)
    assert rc == W.WD_OK
    for dims, U, b, x in keep:
        for k in range(b.shape[0]):
            res = b[k] - oracle.apply_D(x[k], U, dims, 0.13)
            assert np.linalg.norm(res) / np.linalg.norm(b[k]) <= 1.05e-10
    zero = [dict(pr, x=np.zeros_like(pr["b"])) for pr in probs]
    p.use_initial_guess = 0
    rc, fresh = W.wd_solve_batch(zero, p)
    assert rc == W.WD_OK
    assert sum(d["iters"] for d in resumed) < sum(d["iters"] for d in fresh)
