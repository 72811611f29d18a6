"""Python binding of libwd: the same entry points as include/wd.h, by ctypes.

Argument marshalling only.  Buffers may be torch tensors (their data_ptr()
is passed), raw integer addresses, or numpy arrays (host pointers, accepted
where the C entry point accepts host memory, i.e. ``wd_solve``/``wd_solve_ex``).
Every step of the computation runs inside libwd's CUDA kernels; if the
library has not been built, importing functions from here raises.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

WD_F64, WD_F32, WD_F16 = 0, 1, 2
WD_TEMPORAL_GAUGE = 0x100
WD_STAGE_NEIGHBOURS = 0x200
WD_SOLVER_CG, WD_SOLVER_BICGSTAB = 0, 1
WD_EVEN, WD_ODD, WD_FULL = 0, 1, -1

WD_OK = 0
WD_ERR_NULL = 1
WD_ERR_DIMS = 2
WD_ERR_PREC = 3
WD_ERR_ALIGN = 4
WD_ERR_ALIAS = 5
WD_ERR_NOCONV = 6
WD_ERR_NONFINITE = 7
WD_ERR_TIMEOUT = 8
WD_ERR_CUDA = 9
WD_ERR_ARG = 10
WD_ERR_BREAKDOWN = 11
WD_ERR_SCRATCH = 12

# every function declared in include/wd.h
EXPORTS = [
    "wd_set_stream", "wd_get_stream", "wd_error_string", "wd_last_cuda_error", "wd_finalize",
    "wd_spinor_bytes", "wd_gauge_bytes", "wd_pack_gauge", "wd_pack_spinor", "wd_unpack_spinor",
    "wd_convert_spinor", "wd_dslash", "wd_dslash_dag", "wd_dslash_ex", "wd_mhat", "wd_norm2",
    "wd_cdot", "wd_axpby", "wd_solve_params_default", "wd_solve", "wd_solve_ex",
    "wd_dslash_ex_noalloc", "wd_dslash_mrhs", "wd_solve_batch", "wd_gauge_fix_temporal",
    "wd_rotate_spinor", "wd_tc_gemm_bf16", "wd_nn_train_params_default", "wd_nn_init",
    "wd_nn_apply", "wd_nn_train", "wd_solve_fgcr", "wd_nn_layer", "wd_gaussian_spinor",
    "wd_nn_wgrad", "wd_set_autotune", "wd_mrhs_set_lanes", "wd_tune_report",
    "wd_wait_selftest", "wd_set_wait_limit", "wd_async_status", "wd_solve_fcg",
    "wd_set_batch_mode", "wd_dslash_set_block", "wd_nn_apply_ex", "wd_set_launch_overlap",
]

WD_NN_PARAMS = 2304
WD_NN_BF16, WD_NN_EVEN = 1, 2


class WdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.wd_error_string(status).decode() if _lib is not None else str(status)
        if status == WD_ERR_CUDA and _lib is not None:
            msg += f" (cudaError {_lib.wd_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


class wd_solve_params(C.Structure):
    _fields_ = [("inner_prec", C.c_int), ("inner_recon", C.c_int), ("outer_recon", C.c_int),
                ("reliable_interval", C.c_int), ("check_interval", C.c_int),
                ("maxiter", C.c_int), ("use_graph", C.c_int), ("use_initial_guess", C.c_int),
                ("tol", C.c_double), ("gauge_fix", C.c_int), ("solver", C.c_int)]


class wd_batch_problem(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("kappa", C.c_double), ("nrhs", C.c_int),
                ("gauge", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p)]


class wd_nn_train_params(C.Structure):
    _fields_ = [("samples", C.c_int), ("batch", C.c_int), ("epochs", C.c_int),
                ("lr", C.c_float), ("seed", C.c_ulonglong), ("init", C.c_int),
                ("smooth", C.c_int)]


class wd_nn_train_info(C.Structure):
    _fields_ = [("steps", C.c_int), ("loss_first", C.c_double), ("loss_last", C.c_double),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class wd_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("reliable_updates", C.c_int), ("status", C.c_int),
                ("true_residual", C.c_double), ("seconds", C.c_double),
                ("dslash_calls", C.c_double), ("setup_seconds", C.c_double),
                ("iterate_seconds", C.c_double), ("reliable_seconds", C.c_double),
                ("final_seconds", C.c_double), ("fallback_iters", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libwd.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"libwd is not built ({LIB} missing): run __graft_entry__.build() "
                           "on a machine with nvcc; there is no fallback implementation")
    L = C.CDLL(LIB)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.c_void_p
    i4 = C.c_int * 4
    sig = {
        "wd_set_stream": (C.c_int, [vp]),
        "wd_get_stream": (vp, []),
        "wd_error_string": (C.c_char_p, [C.c_int]),
        "wd_last_cuda_error": (C.c_int, []),
        "wd_finalize": (None, []),
        "wd_spinor_bytes": (C.c_size_t, [i4, C.c_int, C.c_int]),
        "wd_gauge_bytes": (C.c_size_t, [i4, C.c_int, C.c_int]),
        "wd_pack_gauge": (C.c_int, [vp, dp, i4, C.c_int, C.c_int]),
        "wd_pack_spinor": (C.c_int, [vp, dp, i4, C.c_int, C.c_int]),
        "wd_unpack_spinor": (C.c_int, [dp, vp, i4, C.c_int, C.c_int]),
        "wd_convert_spinor": (C.c_int, [vp, C.c_int, vp, C.c_int, i4, C.c_int]),
        "wd_dslash": (C.c_int, [vp, vp, vp, C.c_double, C.c_int, i4, C.c_int]),
        "wd_dslash_dag": (C.c_int, [vp, vp, vp, C.c_double, C.c_int, i4, C.c_int]),
        "wd_dslash_ex": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_double, vp, C.c_double,
                                   vp, C.c_double, dp, i4, C.c_int, C.c_int]),
        "wd_dslash_ex_noalloc": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_double, vp,
                                           C.c_double, vp, C.c_double, dp, i4, C.c_int,
                                           C.c_int]),
        "wd_mhat": (C.c_int, [vp, vp, vp, vp, C.c_double, C.c_int, i4, C.c_int, C.c_int]),
        "wd_gauge_fix_temporal": (C.c_int, [dp, dp, dp, i4]),
        "wd_tc_gemm_bf16": (C.c_int, [dp, vp, vp, C.c_int, C.c_int, C.c_int]),
        "wd_nn_train_params_default": (None, [C.POINTER(wd_nn_train_params)]),
        "wd_nn_init": (C.c_int, [dp, C.c_double]),
        "wd_nn_layer": (C.c_int, [vp, vp, dp, C.c_int, C.c_int, vp, i4]),
        "wd_nn_wgrad": (C.c_int, [dp, vp, vp, C.c_int, C.c_int, vp, i4]),
        "wd_gaussian_spinor": (C.c_int, [vp, C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, i4]),
        "wd_nn_apply": (C.c_int, [vp, vp, dp, vp, i4]),
        "wd_nn_apply_ex": (C.c_int, [vp, vp, dp, vp, i4, C.c_int]),
        "wd_nn_train": (C.c_int, [dp, dp, C.c_double, i4, C.POINTER(wd_nn_train_params),
                                  C.POINTER(wd_nn_train_info)]),
        "wd_solve_fgcr": (C.c_int, [dp, dp, dp, C.c_double, i4, dp, C.c_int,
                                    C.POINTER(wd_solve_params), C.POINTER(wd_solve_info)]),
        "wd_rotate_spinor": (C.c_int, [dp, dp, dp, i4, C.c_int]),
        "wd_solve_fcg": (C.c_int, [dp, dp, dp, C.c_double, i4, dp,
                                   C.POINTER(wd_solve_params), C.POINTER(wd_solve_info)]),
        "wd_dslash_mrhs": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_double, vp, C.c_double,
                                     C.c_int, dp, i4, C.c_int, C.c_int]),
        "wd_set_autotune": (C.c_int, [C.c_int]),
        "wd_set_batch_mode": (C.c_int, [C.c_int]),
        "wd_dslash_set_block": (C.c_int, [C.c_int]),
        "wd_set_launch_overlap": (C.c_int, [C.c_int]),
        "wd_wait_selftest": (C.c_int, [C.c_longlong]),
        "wd_set_wait_limit": (C.c_int, [C.c_longlong]),
        "wd_async_status": (C.c_int, []),
        "wd_mrhs_set_lanes": (C.c_int, [C.c_int]),
        "wd_tune_report": (C.c_int, [C.c_char_p, C.c_size_t]),
        "wd_solve_batch": (C.c_int, [C.POINTER(wd_batch_problem), C.c_int,
                                     C.POINTER(wd_solve_params), C.POINTER(wd_solve_info)]),
        "wd_norm2": (C.c_int, [dp, vp, i4, C.c_int, C.c_int]),
        "wd_cdot": (C.c_int, [dp, vp, vp, i4, C.c_int, C.c_int]),
        "wd_axpby": (C.c_int, [C.c_double, vp, C.c_double, vp, i4, C.c_int, C.c_int]),
        "wd_solve_params_default": (None, [C.POINTER(wd_solve_params)]),
        "wd_solve": (C.c_int, [dp, dp, dp, C.c_double, C.c_double, i4]),
        "wd_solve_ex": (C.c_int, [dp, dp, dp, C.c_double, i4, C.POINTER(wd_solve_params),
                                  C.POINTER(wd_solve_info)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _p(t):
    """Address of a buffer: torch tensor, numpy array, int or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def _d(dims):
    return (C.c_int * 4)(*[int(v) for v in dims])


def _ck(rc, where):
    if rc != WD_OK:
        raise WdError(rc, where)


# ---------------------------------------------------------------------------
# entry points (same names and argument order as include/wd.h)
# ---------------------------------------------------------------------------

def wd_set_stream(stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _ck(lib().wd_set_stream(stream), "wd_set_stream")


def wd_get_stream():
    return lib().wd_get_stream()


def wd_error_string(status):
    return lib().wd_error_string(int(status)).decode()


def wd_last_cuda_error():
    return lib().wd_last_cuda_error()


def wd_finalize():
    lib().wd_finalize()


def wd_spinor_bytes(dims, parity, prec):
    return int(lib().wd_spinor_bytes(_d(dims), int(parity), int(prec)))


def wd_gauge_bytes(dims, prec, recon=12):
    return int(lib().wd_gauge_bytes(_d(dims), int(prec), int(recon)))


def wd_pack_gauge(dst, src_canonical, dims, prec, recon=12):
    _ck(lib().wd_pack_gauge(_p(dst), _p(src_canonical), _d(dims), int(prec), int(recon)),
        "wd_pack_gauge")


def wd_pack_spinor(dst, src_canonical, dims, parity, prec):
    _ck(lib().wd_pack_spinor(_p(dst), _p(src_canonical), _d(dims), int(parity), int(prec)),
        "wd_pack_spinor")


def wd_unpack_spinor(dst_canonical, src, dims, parity, prec):
    _ck(lib().wd_unpack_spinor(_p(dst_canonical), _p(src), _d(dims), int(parity), int(prec)),
        "wd_unpack_spinor")


def wd_convert_spinor(dst, dst_prec, src, src_prec, dims, parity):
    _ck(lib().wd_convert_spinor(_p(dst), int(dst_prec), _p(src), int(src_prec), _d(dims),
                                int(parity)), "wd_convert_spinor")


def wd_dslash(out, inp, gauge, kappa, parity, dims, prec):
    _ck(lib().wd_dslash(_p(out), _p(inp), _p(gauge), float(kappa), int(parity), _d(dims),
                        int(prec)), "wd_dslash")


def wd_dslash_dag(out, inp, gauge, kappa, parity, dims, prec):
    _ck(lib().wd_dslash_dag(_p(out), _p(inp), _p(gauge), float(kappa), int(parity), _d(dims),
                            int(prec)), "wd_dslash_dag")


def wd_dslash_ex(out, inp, gauge, parity, dagger, a, x, bx, y, cy, norm2, dims, prec, recon=12):
    _ck(lib().wd_dslash_ex(_p(out), _p(inp), _p(gauge), int(parity), int(dagger), float(a),
                           _p(x), float(bx), _p(y), float(cy), _p(norm2), _d(dims), int(prec),
                           int(recon)), "wd_dslash_ex")


def wd_dslash_ex_noalloc(out, inp, gauge, parity, dagger, a, x, bx, y, cy, norm2, dims, prec,
                         recon=12):
    """wd_dslash_ex without any device allocation (fixed scratch inside libwd;
    V/2 <= 2,097,152 sites).  For callers that cannot let the library call
    cudaMalloc: stream-capturing code, foreign-allocator applications,
    latency-critical loops."""
    _ck(lib().wd_dslash_ex_noalloc(_p(out), _p(inp), _p(gauge), int(parity), int(dagger),
                                   float(a), _p(x), float(bx), _p(y), float(cy), _p(norm2),
                                   _d(dims), int(prec), int(recon)), "wd_dslash_ex_noalloc")


def wd_dslash_mrhs(out, inp, gauge, parity, dagger, a, x, bx, nrhs, norm2, dims, prec, recon=12):
    _ck(lib().wd_dslash_mrhs(_p(out), _p(inp), _p(gauge), int(parity), int(dagger), float(a),
                             _p(x), float(bx), int(nrhs), _p(norm2), _d(dims), int(prec),
                             int(recon)), "wd_dslash_mrhs")


def wd_wait_selftest(spins):
    """Run the bounded-wait failure path on purpose; returns the status
    (WD_ERR_TIMEOUT is the expected answer)."""
    return int(lib().wd_wait_selftest(int(spins)))


def wd_set_wait_limit(polls):
    """Polls of the bounded wait of the asynchronous (staged) kernels."""
    _ck(lib().wd_set_wait_limit(int(polls)), "wd_set_wait_limit")


def wd_async_status():
    """WD_OK, or WD_ERR_TIMEOUT if an asynchronous launch gave up waiting since
    the last call (the flag is cleared); waits for the set stream."""
    rc = int(lib().wd_async_status())
    if rc not in (WD_OK, WD_ERR_TIMEOUT):
        raise WdError(rc, "wd_async_status")
    return rc


def wd_set_batch_mode(mode):
    """0: one launch per step of a batched CG iteration (default); 1: one
    persistent cooperative launch per iteration.  Returns the previous mode."""
    prev = int(lib().wd_set_batch_mode(int(mode)))
    if prev < 0:
        raise WdError(-prev, "wd_set_batch_mode")
    return prev


def wd_set_autotune(enable):
    """Turn the multi-RHS tile-shape autotuner on or off; returns the previous
    setting."""
    return int(lib().wd_set_autotune(int(enable)))


def wd_dslash_set_block(sites):
    """Force the CTA size (64, 128, 256) of the non-reducing single-field
    hopping launches, or return to the tuned sizes (0)."""
    _ck(lib().wd_dslash_set_block(int(sites)), "wd_dslash_set_block")


def wd_set_launch_overlap(enable):
    """Launch the single-field hopping kernels as programmatic dependent
    launches (1, the default) or as plain stream-ordered launches (0); results
    are identical.  Returns the previous setting."""
    return int(lib().wd_set_launch_overlap(int(enable)))


def wd_mrhs_set_lanes(lanes):
    """Force the multi-RHS tile shape or return to the tuned shapes (0).  Shape
    codes: 1, 2, 4, 8 right-hand-side warps per CTA with one right-hand side
    per thread; 17, 18, 20 = 16 + warps with two per thread (FP32)."""
    _ck(lib().wd_mrhs_set_lanes(int(lanes)), "wd_mrhs_set_lanes")


def wd_tune_report():
    """(number of tuned shapes, text table)."""
    n = int(lib().wd_tune_report(None, 0))
    buf = C.create_string_buffer(256 * (n + 1))
    n = int(lib().wd_tune_report(buf, len(buf)))
    return n, buf.value.decode()


def wd_solve_batch(problems, params=None, check=True):
    """problems: list of dicts with dims, kappa, nrhs, gauge, b, x (buffers as
    accepted by _p: host numpy arrays or device tensors).  Returns the status
    and one info dict per right-hand side."""
    n = len(problems)
    arr = (wd_batch_problem * n)()
    for j, pr in enumerate(problems):
        arr[j].dims = (C.c_int * 4)(*[int(v) for v in pr["dims"]])
        arr[j].kappa = float(pr["kappa"])
        arr[j].nrhs = int(pr["nrhs"])
        arr[j].gauge = _p(pr["gauge"])
        arr[j].b = _p(pr["b"])
        arr[j].x = _p(pr["x"])
    nr = sum(int(pr["nrhs"]) for pr in problems)
    infos = (wd_solve_info * max(nr, 1))()
    p = params if params is not None else wd_solve_params_default()
    rc = lib().wd_solve_batch(arr, n, C.byref(p), infos)
    out = [infos[i].as_dict() for i in range(nr)]
    if check:
        _ck(rc, "wd_solve_batch")
    return rc, out


def wd_tc_gemm_bf16(D, A, B, M, K, N):
    _ck(lib().wd_tc_gemm_bf16(_p(D), _p(A), _p(B), int(M), int(K), int(N)), "wd_tc_gemm_bf16")


def wd_nn_train_params_default():
    p = wd_nn_train_params()
    lib().wd_nn_train_params_default(C.byref(p))
    return p


def wd_nn_layer(out, inp, weights, cin, cout, gauge, dims):
    _ck(lib().wd_nn_layer(_p(out), _p(inp), _p(weights), int(cin), int(cout), _p(gauge), _d(dims)),
        "wd_nn_layer")


def wd_nn_wgrad(grad, inp, delta, cin, cout, gauge, dims):
    _ck(lib().wd_nn_wgrad(_p(grad), _p(inp), _p(delta), int(cin), int(cout), _p(gauge), _d(dims)),
        "wd_nn_wgrad")


def wd_gaussian_spinor(out, seed, stream, first, dims):
    _ck(lib().wd_gaussian_spinor(_p(out), int(seed), int(stream), int(first), _d(dims)),
        "wd_gaussian_spinor")


def nn_field_bytes(dims, channels):
    """Bytes of a packed FP32 full field with `channels` channels per colour."""
    vh = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3]) // 2
    vh_pad = (vh + 31) // 32 * 32
    return 2 * ((vh_pad * channels * 24 + 255) // 256 * 256)


def wd_nn_init(weights, kappa):
    _ck(lib().wd_nn_init(_p(weights), float(kappa)), "wd_nn_init")


def wd_nn_apply(out, inp, weights, gauge, dims):
    _ck(lib().wd_nn_apply(_p(out), _p(inp), _p(weights), _p(gauge), _d(dims)), "wd_nn_apply")


def wd_nn_apply_ex(out, inp, weights, gauge, dims, flags=0):
    """out = N(inp); flags: WD_NN_BF16 (BF16 activations), WD_NN_EVEN (the
    even-even block only)."""
    _ck(lib().wd_nn_apply_ex(_p(out), _p(inp), _p(weights), _p(gauge), _d(dims), int(flags)),
        "wd_nn_apply_ex")


def wd_nn_train(weights, gauge, kappa, dims, params=None):
    p = params if params is not None else wd_nn_train_params_default()
    info = wd_nn_train_info()
    _ck(lib().wd_nn_train(_p(weights), _p(gauge), float(kappa), _d(dims), C.byref(p),
                          C.byref(info)), "wd_nn_train")
    return info.as_dict()


def wd_solve_fgcr(x, b, gauge, kappa, dims, weights=None, m=10, params=None, check=True):
    info = wd_solve_info()
    p = params if params is not None else wd_solve_params_default()
    rc = lib().wd_solve_fgcr(_p(x), _p(b), _p(gauge), float(kappa), _d(dims), _p(weights), int(m),
                             C.byref(p), C.byref(info))
    out = info.as_dict()
    out["status"] = rc
    if check:
        _ck(rc, "wd_solve_fgcr")
    return out


def wd_solve_fcg(x, b, gauge, kappa, dims, weights=None, params=None, check=True):
    """Flexible CG on D^+ D x = D^+ b preconditioned by N N^+ (weights None:
    plain CGNR); plain even-odd CG is the fallback.  Returns the info dict."""
    info = wd_solve_info()
    p = params if params is not None else wd_solve_params_default()
    rc = lib().wd_solve_fcg(_p(x), _p(b), _p(gauge), float(kappa), _d(dims), _p(weights),
                            C.byref(p), C.byref(info))
    out = info.as_dict()
    out["status"] = rc
    if check:
        _ck(rc, "wd_solve_fcg")
    return out


def wd_gauge_fix_temporal(U_out, omega_out, U_in, dims):
    _ck(lib().wd_gauge_fix_temporal(_p(U_out), _p(omega_out), _p(U_in), _d(dims)),
        "wd_gauge_fix_temporal")


def wd_rotate_spinor(out, inp, omega, dims, dagger=0):
    _ck(lib().wd_rotate_spinor(_p(out), _p(inp), _p(omega), _d(dims), int(dagger)),
        "wd_rotate_spinor")


def wd_mhat(out, inp, gauge, tmp, kappa, dagger, dims, prec, recon=12):
    _ck(lib().wd_mhat(_p(out), _p(inp), _p(gauge), _p(tmp), float(kappa), int(dagger), _d(dims),
                      int(prec), int(recon)), "wd_mhat")


def wd_norm2(result, x, dims, parity, prec):
    _ck(lib().wd_norm2(_p(result), _p(x), _d(dims), int(parity), int(prec)), "wd_norm2")


def wd_cdot(result, x, y, dims, parity, prec):
    _ck(lib().wd_cdot(_p(result), _p(x), _p(y), _d(dims), int(parity), int(prec)), "wd_cdot")


def wd_axpby(a, x, b, y, dims, parity, prec):
    _ck(lib().wd_axpby(float(a), _p(x), float(b), _p(y), _d(dims), int(parity), int(prec)),
        "wd_axpby")


def wd_solve_params_default():
    p = wd_solve_params()
    lib().wd_solve_params_default(C.byref(p))
    return p


def wd_solve(x, b, gauge, kappa, tol, dims):
    _ck(lib().wd_solve(_p(x), _p(b), _p(gauge), float(kappa), float(tol), _d(dims)), "wd_solve")


def wd_solve_ex(x, b, gauge, kappa, dims, params=None, check=True):
    """Returns the wd_solve_info as a dict (status included); raises on a
    non-zero status unless check=False."""
    info = wd_solve_info()
    p = params if params is not None else wd_solve_params_default()
    rc = lib().wd_solve_ex(_p(x), _p(b), _p(gauge), float(kappa), _d(dims), C.byref(p),
                           C.byref(info))
    out = info.as_dict()
    out["status"] = rc
    if check:
        _ck(rc, "wd_solve_ex")
    return out


# ---------------------------------------------------------------------------
# buffer helpers (torch owns the memory; sizes come from libwd)
# ---------------------------------------------------------------------------

def alloc_spinor(dims, parity, prec, device="cuda"):
    """Uninitialised packed spinor buffer (torch uint8 tensor)."""
    import torch
    n = wd_spinor_bytes(dims, parity, prec)
    if n == 0:
        raise WdError(WD_ERR_ARG, "alloc_spinor")
    return torch.empty(n, dtype=torch.uint8, device=device)


def alloc_gauge(dims, prec, recon=12, device="cuda"):
    """Uninitialised packed gauge buffer (torch uint8 tensor)."""
    import torch
    n = wd_gauge_bytes(dims, prec, recon)
    if n == 0:
        raise WdError(WD_ERR_PREC, "alloc_gauge")
    return torch.empty(n, dtype=torch.uint8, device=device)
