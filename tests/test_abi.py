"""CPU-only checks of the C ABI: the library builds, loads, exports every
symbol that include/wd.h declares, and its host-side validation answers
without touching a GPU (every case below fails validation before any CUDA
call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def W():
    from paper_0810_5365_gb300 import build as B
    B.build()
    import paper_0810_5365_gb300 as W
    W.wd.lib()
    return W


def header_functions():
    text = open(os.path.join(ROOT, "include", "wd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_dslash_and_solve_calls():
    fns = header_functions()
    for name in ("wd_dslash", "wd_solve", "wd_dslash_dag", "wd_solve_ex", "wd_pack_gauge",
                 "wd_pack_spinor", "wd_unpack_spinor", "wd_set_stream", "wd_finalize"):
        assert name in fns


def test_every_declared_symbol_is_exported(W):
    L = W.wd.lib()
    fns = header_functions()
    assert fns, "no declarations parsed"
    for name in fns:
        assert hasattr(L, name), name
    assert sorted(W.wd.EXPORTS) == fns


def test_sizes(W):
    d = (4, 4, 4, 4)
    Vh = 128
    assert W.wd_spinor_bytes(d, W.WD_EVEN, W.WD_F64) == Vh * 192
    assert W.wd_spinor_bytes(d, W.WD_ODD, W.WD_F32) == Vh * 96
    assert W.wd_spinor_bytes(d, W.WD_FULL, W.WD_F32) == 2 * Vh * 96
    assert W.wd_spinor_bytes(d, W.WD_EVEN, W.WD_F16) == Vh * 52
    assert W.wd_gauge_bytes(d, W.WD_F32, 12) == 8 * Vh * 48
    assert W.wd_gauge_bytes(d, W.WD_F64, 18) == 8 * Vh * 144
    assert W.wd_gauge_bytes(d, W.WD_F16, 12) == 8 * Vh * 24
    # ragged: Vh = 6*6*6*6/2 = 648 is padded to 672 (a multiple of 32), then to 256 B
    d2 = (6, 6, 6, 6)
    assert W.wd_spinor_bytes(d2, W.WD_EVEN, W.WD_F32) == 672 * 96
    assert W.wd_spinor_bytes(d2, W.WD_EVEN, W.WD_F16) == (672 * 52 + 255) // 256 * 256


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 0), (4, 1, 4, 4), (4, 4, 4, 5)])
def test_bad_dims_rejected(W, dims):
    assert W.wd_spinor_bytes(dims, 0, W.WD_F32) == 0
    with pytest.raises(W.WdError) as e:
        W.wd_dslash(16, 32, 48, 0.1, 0, dims, W.WD_F32)
    assert e.value.status == W.WD_ERR_DIMS


def test_bad_precision_and_recon(W):
    d = (4, 4, 4, 4)
    assert W.wd_gauge_bytes(d, W.WD_F16, 18) == 0
    assert W.wd_gauge_bytes(d, 7, 12) == 0
    with pytest.raises(W.WdError) as e:
        W.wd_dslash(16, 32, 48, 0.1, 0, d, 5)
    assert e.value.status == W.WD_ERR_PREC
    with pytest.raises(W.WdError) as e:
        W.wd_dslash_ex(16, 32, 48, 0, 0, 1.0, None, 0, None, 0, None, d, W.WD_F16, 18)
    assert e.value.status == W.WD_ERR_PREC


def test_null_alias_align_parity(W):
    d = (4, 4, 4, 4)
    with pytest.raises(W.WdError) as e:
        W.wd_dslash(None, 32, 48, 0.1, 0, d, W.WD_F32)
    assert e.value.status == W.WD_ERR_NULL
    with pytest.raises(W.WdError) as e:
        W.wd_dslash(32, 32, 48, 0.1, 0, d, W.WD_F32)
    assert e.value.status == W.WD_ERR_ALIAS
    with pytest.raises(W.WdError) as e:
        W.wd_dslash(16, 40, 48, 0.1, 0, d, W.WD_F32)
    assert e.value.status == W.WD_ERR_ALIGN
    with pytest.raises(W.WdError) as e:
        W.wd_dslash_ex(16, 32, 48, 2, 0, 1.0, None, 0, None, 0, None, d, W.WD_F32, 12)
    assert e.value.status == W.WD_ERR_ARG
    with pytest.raises(W.WdError) as e:
        W.wd_mhat(16, 32, 48, 32, 0.1, 0, d, W.WD_F32, 12)
    assert e.value.status == W.WD_ERR_ALIAS


def test_error_strings(W):
    for s in range(13):
        assert W.wd_error_string(s).startswith("WD_")
    assert W.wd_error_string(999) == "unknown status"


def test_solve_params_default(W):
    p = W.wd_solve_params_default()
    assert p.inner_prec == W.WD_F32 and p.reliable_interval == 50 and p.tol == 1e-10
    assert p.outer_recon == 18 and p.inner_recon == 12 and p.use_graph == 1


def test_product_path_has_no_oracle_or_fallback():
    """The CUDA path never imports the oracle, and there is no CPU fallback."""
    pkg = os.path.join(ROOT, "paper_0810_5365_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower() or f == "build.py", f
                assert "import synth" not in text and "from synth" not in text, f


def test_stream_and_error_state_roundtrip(W):
    """wd_set_stream / wd_get_stream keep the handle they were given, and
    wd_last_cuda_error starts at 0 (host state only; no CUDA call)."""
    prev = W.wd_get_stream()
    W.wd_set_stream(0x1234)
    assert W.wd_get_stream() == 0x1234
    W.wd_set_stream(prev)
    assert W.wd_get_stream() == prev
    assert W.wd_last_cuda_error() == 0


def test_tuner_controls_on_host(W):
    """The autotuner switches and report answer on the host: the setting
    round-trips, only the shape codes 0, 1, 2, 4, 8 (one right-hand side per
    thread) and 17, 18, 20 (two) are accepted, and the report has one line per
    tuned shape (none when no GPU test ran before in this process)."""
    prev = W.wd_set_autotune(0)
    assert W.wd_set_autotune(prev) == 0
    for lanes in (1, 2, 4, 8, 17, 18, 20, 0):
        W.wd_mrhs_set_lanes(lanes)
    for bad in (-1, 3, 16, 24, 25):
        with pytest.raises(W.WdError):
            W.wd_mrhs_set_lanes(bad)
    n, text = W.wd_tune_report()
    assert n >= 0 and len(text.splitlines()) == n


def test_batch_limits_rejected_on_host(W):
    """wd_solve_batch takes 1..16 problems of 1..32 right-hand sides each;
    anything else is WD_ERR_ARG before any CUDA call."""
    import numpy as np
    dims = (4, 4, 4, 4)
    V = 256
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)

    def prob(nrhs):
        b = np.zeros((nrhs, V, 4, 3), dtype=np.complex128)
        return {"dims": dims, "kappa": 0.12, "nrhs": nrhs, "gauge": U, "b": b,
                "x": np.zeros_like(b)}

    rc, _ = W.wd_solve_batch([prob(33)], check=False)
    assert rc == W.WD_ERR_ARG
    rc, _ = W.wd_solve_batch([prob(0 + 1)] * 17, check=False)
    assert rc == W.WD_ERR_ARG
