"""Benchmark: even-odd Wilson dslash throughput on a 32^3x64 lattice, and
time-to-solution of the solvers built on it.

Headline: one step = one parity-restricted hopping application (Dslash of
the paper's section "Wilson inverter: Main features") over the
V/2 = 1,048,576 sites of one parity, FP32 with 12-real links, alternating the
output parity each step.  Effective Gflops use the nominal 1320 flops per
site (reconstruction work not counted, as the paper counts its effective
Gflops, section "Performance").

The JSON line (rank 0) carries, besides metric/value/unit:
  roofline      achieved GB/s against the measured copy peak (and the nominal
                8 TB/s), with the DRAM traffic per launch from the committed
                ncu counters while the kernel sources are unchanged;
  graph         the same launches captured as one CUDA graph;
  mhat          the even-odd operator 1 - kappa^2 D_eo D_oe (the paper's Fig. 1);
  variants      FP16, FP64, the temporal-gauge variants and the FP16 kernel with
                TMA-staged far neighbours;
  e2e           the headline through the C ABI with pinned host buffers and
                the copies inside the timed region (pipelined over streams);
  clocks        SM clocks and throttle reasons sampled during the timing;
  summary       the figures of the sections below in a few short keys;
  cpu_baseline  the FP64 oracle on the host cores (and one thread), plus the
                oracle's plain FP64 CG to 1e-10 on 24^3x48, timed whole;
  solve         time to a 1e-10 true residual on 24^3x48: mixed-precision CG
                and BiCGstab against plain FP64 CG;
  batch         batched multi-right-hand-side solves against the same solves
                one at a time, and the autotuner's tile shapes;
  learned_preconditioner  training at kappa = 0.137, and even-odd flexible CG
                with the preconditioner N_e N_e^+ (trained network, untrained
                series, none)
                against plain FP64 CG and mixed CG on 16^3x32 and 32^3x64.
``--impl reference`` times the FP64 CPU oracle on the same workload instead
(bounded sample per step).  ``--profile NAME`` runs a short fixed workload for
an ncu capture.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "dslash GB/s & Gflops vs HBM peak; time-to-1e-10 solve vs plain FP64 CG"
FLOPS_PER_SITE = 1320
# compulsory bytes per output site of one parity application: 8 links, the
# input spinor once, the output spinor once
BYTES_PER_SITE = {"f32": 8 * 48 + 96 + 96, "f16": 8 * 24 + 52 + 52, "f64": 8 * 144 + 192 + 192}
DIMS = (32, 32, 32, 64)
KAPPA = 0.1365
DATA = ("synthetic: seeded SU(3) links U = reunit(exp(i 0.3 H)), H Gaussian traceless "
        "Hermitian; complex-Gaussian spinor (no dataset or checkpoint)")


def dslash_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0810_5365_gb300", "csrc")
    for f in ("wd_common.cuh", "wd_dslash.cuh", "wd_internal.h", "wd_dslash_f32.cu",
              "wd_dslash_f16.cu", "wd_dslash_f64.cu", "wd_dslash_staged.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def tg_bytes_per_site(name, dims):
    """Algorithmic bytes per output site in temporal gauge: the two time links
    are read only by the sites next to the boundary slice (1/L3 of them)."""
    link = {"f32_tg": 48, "f16_tg": 24}[name]
    spin = {"f32_tg": 96, "f16_tg": 52}[name]
    return 6 * link + 2 * link / dims[3] + 2 * spin


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def profiled_traffic(prec: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "dslash_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except OSError:
        return None
    e = d.get(prec)
    if not e or e.get("source_hash") != dslash_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle samples in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=self.file,
                stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.file.flush()
        with open(self.file.name) as f:
            rows = [r.strip().split(",") for r in f if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def make_fields(dims):
    from synth import fields
    U = fields.su3_links(dims)
    psi = fields.gaussian_spinor(dims)
    return U, psi


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# the CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_step_sample(U, psi, dims, target_s=0.05):
    """Pick a site sample so one oracle step takes about target_s seconds."""
    import oracle
    from synth import fields
    sites = fields.half_sites(dims, 0)
    n = 4096
    t0 = time.perf_counter()
    oracle.hop_sites(psi, U, dims, sites[:n])
    dt = time.perf_counter() - t0
    n = int(min(len(sites), max(1024, n * target_s / max(dt, 1e-6))))
    return sites[:n]


def cpu_baseline(U, psi, dims, budget_s=12.0):
    """The FP64 oracle's parity dslash on the same fields, on all host cores,
    repeated over whole-lattice applications until about budget_s of work."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    Vh = int(np.prod(dims)) // 2
    n, t = 0, 0.0
    while t < budget_s and n < 400:
        t0 = time.perf_counter()
        oracle.hop(psi, U, dims, dagger=False, out_parity=0)
        t += time.perf_counter() - t0
        n += 1
    out = {"value": FLOPS_PER_SITE * Vh * n / t / 1e9, "unit": "Gflops",
           "cores": oracle.get_threads(), "kind": "oracle",
           "sample": f"{n} full even-parity applications of the FP64 oracle hopping term "
                     f"on the 32^3x64 fields ({t:.1f} s)"}
    # one thread, on a slice of the same fields (every 128th site)
    sites = np.arange(0, Vh * 2, 128)
    oracle.set_threads(1)
    n1, t1 = 0, 0.0
    while t1 < 2.0:
        t0 = time.perf_counter()
        oracle.hop_sites(psi, U, dims, sites)
        t1 += time.perf_counter() - t0
        n1 += 1
    oracle.set_threads(cores)
    out["single_thread_gflops"] = FLOPS_PER_SITE * len(sites) * n1 / t1 / 1e9
    return out


def oracle_cg_full(maxiter=4000):
    """Plain FP64 CG of the oracle (CG on D^+ D of the full lattice, two D
    applications per iteration, all host cores) on the 24^3x48 solve problem
    of the GPU's solve comparison, run to a 1e-10 true residual and timed."""
    import oracle
    from synth import fields
    oracle.set_threads(os.cpu_count() or 1)
    U = fields.su3_links(SOLVE_DIMS)
    b = fields.gaussian_spinor(SOLVE_DIMS, seed=2025)
    t0 = time.perf_counter()
    _, its, rel, ok = oracle.cgnr(b, U, SOLVE_DIMS, SOLVE_KAPPA, 1e-10, maxiter)
    dt = time.perf_counter() - t0
    return {"wall_s": dt, "iterations": its, "true_residual": rel, "converged": bool(ok),
            "cores": oracle.get_threads(), "kind": "measured",
            "problem": "24^3x48, kappa 0.137, complex Gaussian b (seed 2025), tol 1e-10"}


def compact_summary(line):
    """The figures of the sub-sections in a few short keys, so that they sit
    near the start of the JSON line."""
    sm = {"dslash_f32_frac": round(line["roofline"]["frac"], 3),
          "variants_frac": {k: round(v["frac"], 3) for k, v in line["variants"].items()},
          "variants_us": {k: round(v["ms_per_step"] * 1e3, 1) for k, v in line["variants"].items()}}
    if "solve" in line:
        sm["solve_24x48_s_iters_speedup"] = {
            k: [round(v["wall_s"], 4), v["iters"], round(v.get("speedup_vs_f64", 1.0), 2)]
            for k, v in line["solve"].items() if k != "config"}
    if "batch" in line:
        bt = line["batch"]
        sm["batch_s_vs_sequential_vs_f64"] = {
            f"{k}_{inner}": [round(v["batched"][inner]["wall_s"], 4),
                             round(v["batched"][inner]["speedup_vs_sequential_same_inner"], 2),
                             round(v["batched"][inner]["speedup_vs_plain_f64"], 2),
                             round(v["batched"][inner]["persistent_launch_wall_s"], 4)]
            for k, v in bt.items() if isinstance(v, dict) and "batched" in v
            for inner in v["batched"]}
        if "mrhs_dslash" in bt:
            sm["mrhs_dslash_12rhs_24x48"] = {"us": round(bt["mrhs_dslash"]["us_per_launch"], 1),
                                             "gbs": round(bt["mrhs_dslash"]["gbs"], 0)}
    if "learned_preconditioner" in line:
        lp = line["learned_preconditioner"]
        sm["learned_k137_s_iters"] = {
            d: {k: [round(v["wall_s"], 4), v["iters"]] for k, v in r.items()}
            for d, r in lp.items() if d not in ("training", "config")}
        sm["learned_training"] = {k: lp["training"][k] for k in ("loss_first", "loss_last",
                                                                 "wall_s")}
    if "cpu_baseline" in line and "oracle_cg_24x24x24x48" in line["cpu_baseline"]:
        oc = line["cpu_baseline"]["oracle_cg_24x24x24x48"]
        sm["oracle_cg_24x48_s_iters"] = [round(oc["wall_s"], 1), oc["iterations"]]
    return sm


def headline_config(dims, world):
    """The workload both arms report."""
    return {"workload": "even-odd dslash 32^3x64, FP32, 12-real links, kappa=0.1365, "
                        "single RHS, parity alternating per step",
            "dims": list(dims), "kappa": KAPPA, "sites_per_step": int(np.prod(dims)) // 2,
            "flops_per_site": FLOPS_PER_SITE,
            "l2": "inputs larger than L2 (links 403 MB + spinors 2 x 101 MB vs 129 MB L2)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    dims = DIMS
    U, psi = make_fields(dims)
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    sites = oracle_step_sample(U, psi, dims)
    for _ in range(args.warmup):
        oracle.hop_sites(psi, U, dims, sites)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.hop_sites(psi, U, dims, sites)
    dt = time.perf_counter() - t0
    value = FLOPS_PER_SITE * len(sites) * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gflops",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": DATA,
        "config": headline_config(dims, world),
        "cpu_baseline": {"value": value, "unit": "Gflops", "cores": oracle.get_threads(),
                         "kind": "oracle",
                         "sample": f"{len(sites)} even sites of the 32^3x64 fields per step "
                                   "(FP64 oracle hopping term, all host cores)"},
        "e2e": {"value": value, "unit": "Gflops", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU path
# ---------------------------------------------------------------------------

def time_dslash(W, torch, prec_id, recon, gauge, bufs, dims, steps, warmup, stream):
    """K back-to-back parity dslash launches (ping-pong), CUDA events on the
    launching stream.  Returns elapsed seconds."""
    a, b = bufs

    def step(k):
        if k & 1:
            W.wd_dslash_ex(a, b, gauge, W.WD_ODD, 0, -KAPPA, None, 0.0, None, 0.0, None, dims,
                           prec_id, recon)
        else:
            W.wd_dslash_ex(b, a, gauge, W.WD_EVEN, 0, -KAPPA, None, 0.0, None, 0.0, None, dims,
                           prec_id, recon)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        step(k)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def time_dslash_graph(W, torch, gauge, bufs, dims, steps):
    """The same K back-to-back FP32 launches captured once as a CUDA graph and
    replayed (one host launch for all K).  Returns elapsed seconds."""
    a, b = bufs
    cap = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    W.wd_set_stream(cap)
    try:
        with torch.cuda.graph(graph, stream=cap):
            for k in range(steps):
                if k & 1:
                    W.wd_dslash_ex(a, b, gauge, W.WD_ODD, 0, -KAPPA, None, 0.0, None, 0.0, None,
                                   dims, W.WD_F32, 12)
                else:
                    W.wd_dslash_ex(b, a, gauge, W.WD_EVEN, 0, -KAPPA, None, 0.0, None, 0.0,
                                   None, dims, W.WD_F32, 12)
    finally:
        W.wd_set_stream(torch.cuda.current_stream())
    graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    graph.replay()
    e1.record(st)
    e1.synchronize()
    del graph
    return e0.elapsed_time(e1) / 1e3


def max_over_ranks(seconds: float, device: str) -> float:
    """Replicas report the slowest rank's time (the job ends when it does);
    a barrier follows so that no rank starts the next phase early."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest time."""
    return units_per_rank * world / seconds


SOLVE_DIMS = (24, 24, 24, 48)
SOLVE_KAPPA = 0.1370
# BiCGstab works on the non-Hermitian Schur operator itself; on these links
# its spectrum encloses the origin near kappa = 0.137 (FP64 BiCGstab on the CPU
# breaks down there too), so the BiCGstab comparison runs at kappa = 0.130
SOLVE_KAPPA_NONSYM = 0.1300


def solve_section(W, torch, reps=3):
    """Time to a 1e-10 true residual on 24^3x48, kappa = 0.137: mixed
    precision CG (FP16 / FP32 inner, FP64 reliable updates every 50; also in
    temporal gauge) against plain FP64 CG (the same even-odd CGLS, all FP64),
    on the same GPU; and, at kappa = 0.130, mixed-precision BiCGstab against
    plain FP64 CG and mixed CG at that kappa.
    Device-resident canonical inputs; one warm-up solve per precision; the
    median of `reps` timed solves.  Also one solve from host (numpy) buffers
    per precision, copies included."""
    from synth import fields
    dims = SOLVE_DIMS
    U = fields.su3_links(dims)
    b = fields.gaussian_spinor(dims, seed=2025)
    Ud = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    bd = torch.from_numpy(b.view(np.float64).reshape(-1)).cuda()
    x = torch.zeros_like(bd)
    xh = np.zeros_like(b)
    out = {}
    Vh = int(np.prod(dims)) // 2
    k2 = SOLVE_KAPPA_NONSYM
    runs_spec = (("f16", W.WD_F16, 0, 0, SOLVE_KAPPA), ("f32", W.WD_F32, 0, 0, SOLVE_KAPPA),
                 ("f64", W.WD_F64, 0, 0, SOLVE_KAPPA),
                 ("f16_gauge_fixed", W.WD_F16, 1, 0, SOLVE_KAPPA),
                 ("k130_f64", W.WD_F64, 0, 0, k2), ("k130_f16", W.WD_F16, 0, 0, k2),
                 ("k130_f16_bicgstab", W.WD_F16, 0, 1, k2),
                 ("k130_f32_bicgstab", W.WD_F32, 0, 1, k2),
                 ("k130_f16_bicgstab_gauge_fixed", W.WD_F16, 1, 1, k2))
    for name, inner, gf, sv, kappa in runs_spec:
        p = W.wd_solve_params_default()
        p.inner_prec = inner
        p.gauge_fix = gf
        p.solver = sv
        p.maxiter = 100000
        runs = []
        for r in range(reps + 1):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = W.wd_solve_ex(x, bd, Ud, kappa, dims, p, check=False)
            torch.cuda.synchronize()
            info["wall_s"] = time.perf_counter() - t0
            if r > 0:
                runs.append(info)
        runs.sort(key=lambda d: d["wall_s"])
        med = runs[len(runs) // 2]
        xh[:] = 0
        t0 = time.perf_counter()
        ih = W.wd_solve_ex(xh, b, U, kappa, dims, p, check=False)
        host_wall = time.perf_counter() - t0
        out[name] = {
            "kappa": kappa, "solver": "bicgstab" if sv else "cg",
            "wall_s": med["wall_s"], "iters": med["iters"],
            "reliable_updates": med["reliable_updates"], "status": med["status"],
            "true_residual": med["true_residual"],
            "phase_s": {k: med[k] for k in ("setup_seconds", "iterate_seconds",
                                             "reliable_seconds", "final_seconds")},
            "dslash_calls": med["dslash_calls"],
            "dslash_gflops_in_solve": FLOPS_PER_SITE * Vh * med["dslash_calls"]
            / med["wall_s"] / 1e9,
            "host_buffers_wall_s": host_wall, "host_buffers_status": ih["status"],
            "all_wall_s": [d["wall_s"] for d in runs],
        }
    for name in out:
        base = "k130_f64" if name.startswith("k130_") else "f64"
        if name != base:
            out[name]["speedup_vs_f64"] = out[base]["wall_s"] / out[name]["wall_s"]
    out["config"] = {"dims": list(dims), "kappa": SOLVE_KAPPA, "kappa_k130": k2, "tol": 1e-10,
                     "rhs": "complex Gaussian (seed 2025)", "links": "eps=0.3, seed 1234",
                     "reliable_interval": 50, "timing": f"median of {reps} after 1 warm-up"}
    return out


BATCH_KAPPA = 0.1360


def batch_section(W, torch):
    """Batched multi-right-hand-side solves (FP32 and FP16 inner, FP64
    reliable updates, 1e-10 true residual):
    (a) 12 point sources (one per spin-colour index at the origin) on 24^3x48;
    (b) a mixed batch, 4 Gaussian right-hand sides on each of 8^4, 16^3x32
        and 24^3x48 -- one batched launch per step for all 12;
    each against the same right-hand sides solved one at a time with the
    single-right-hand-side mixed solver and with plain FP64 CG, plus the
    multi-RHS hopping kernel's throughput (12 right-hand sides, 24^3x48)."""
    from synth import fields
    out = {}

    def run_batch(spec, name):
        probs, singles = [], []
        for dims, nrhs, kind, seed in spec:
            U = fields.su3_links(dims, seed=seed)
            if kind == "point":
                bs = [fields.point_source(dims, 0, r // 3, r % 3) for r in range(nrhs)]
            else:
                bs = [fields.gaussian_spinor(dims, seed=seed + 1 + r) for r in range(nrhs)]
            b = torch.from_numpy(np.ascontiguousarray(np.stack(bs)).view(np.float64)).cuda()
            Ud = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
            probs.append({"dims": dims, "kappa": BATCH_KAPPA, "nrhs": nrhs, "gauge": Ud, "b": b,
                          "x": torch.zeros_like(b)})
        batched = {}
        for label, inner in (("f32", W.WD_F32), ("f16", W.WD_F16)):
            p = W.wd_solve_params_default()
            p.inner_prec = inner
            per_mode = {}
            # mode 0: one launch per step, a graph of check_interval iterations
            # (the default); mode 1: one persistent launch per iteration
            for mode in (0, 1):
                prev = W.wd_set_batch_mode(mode)
                try:
                    W.wd_solve_batch(probs, p, check=False)  # warm-up
                    for pr in probs:
                        pr["x"].zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    rc, infos = W.wd_solve_batch(probs, p, check=False)
                    torch.cuda.synchronize()
                    per_mode[mode] = {"status": rc, "wall_s": time.perf_counter() - t0,
                                      "iters": [d["iters"] for d in infos],
                                      "max_true_residual": max(d["true_residual"]
                                                               for d in infos)}
                finally:
                    W.wd_set_batch_mode(prev)
                for pr in probs:
                    pr["x"].zero_()
            batched[label] = per_mode[0]
            batched[label]["persistent_launch_wall_s"] = per_mode[1]["wall_s"]
            batched[label]["persistent_launch_status"] = per_mode[1]["status"]
            batched[label]["persistent_launch_iters"] = per_mode[1]["iters"]
        seq = {}
        for label, inner in (("single_rhs_f32", W.WD_F32), ("single_rhs_f16", W.WD_F16),
                             ("plain_f64", W.WD_F64)):
            q = W.wd_solve_params_default()
            q.inner_prec = inner
            tot, its, worst = 0.0, [], 0.0
            for pr in probs:
                n = pr["nrhs"]
                flat = pr["b"].reshape(-1)
                fl = flat.numel() // n
                assert fl * n == flat.numel() and fl == int(np.prod(pr["dims"])) * 24
                x = torch.zeros(fl, dtype=torch.float64, device="cuda")
                W.wd_solve_ex(x, flat[:fl], pr["gauge"], BATCH_KAPPA, pr["dims"], q,
                              check=False)  # warm-up of this shape
                for r in range(n):
                    x.zero_()
                    rhs = flat[r * fl:(r + 1) * fl]
                    assert rhs.numel() == fl
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    i = W.wd_solve_ex(x, rhs, pr["gauge"], BATCH_KAPPA, pr["dims"], q,
                                      check=False)
                    torch.cuda.synchronize()
                    tot += time.perf_counter() - t0
                    its.append(i["iters"])
                    worst = max(worst, i["true_residual"])
            seq[label] = {"wall_s": tot, "iters": its, "max_true_residual": worst}
        for label in batched:
            t_batch = batched[label]["wall_s"]
            batched[label]["speedup_vs_sequential_same_inner"] = (
                seq["single_rhs_" + label]["wall_s"] / t_batch)
            batched[label]["speedup_vs_plain_f64"] = seq["plain_f64"]["wall_s"] / t_batch
        out[name] = {
            "batched": batched, "sequential": seq,
            "problems": [{"dims": list(d), "nrhs": n, "rhs": k} for d, n, k, _ in spec],
        }
        del probs

    run_batch([((24, 24, 24, 48), 12, "point", 1234)], "point_sources_24x48")
    run_batch([((8, 8, 8, 8), 4, "gauss", 1234), ((16, 16, 16, 32), 4, "gauss", 2234),
               ((24, 24, 24, 48), 4, "gauss", 3234)], "mixed_lattices")

    # the tile shapes the autotuner chose for the batches above
    out["autotune"] = W.wd_tune_report()[1].splitlines()

    # the multi-RHS hopping kernel alone: 12 right-hand sides on 24^3x48
    dims = (24, 24, 24, 48)
    Vh = int(np.prod(dims)) // 2
    U = fields.su3_links(dims)
    Ud = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    g = W.alloc_gauge(dims, W.WD_F32, 12)
    W.wd_pack_gauge(g, Ud, dims, W.WD_F32, 12)
    nr = 12
    h = W.wd_spinor_bytes(dims, 0, W.WD_F32)
    a = torch.zeros(nr * h, dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    src = torch.from_numpy(fields.gaussian_spinor(dims, nsites=Vh).view(np.float64)
                           .reshape(-1)).cuda()
    for r in range(nr):
        W.wd_pack_spinor(a[r * h:(r + 1) * h], src, dims, 1, W.WD_F32)
    n_steps = 200
    for k in range(10):
        W.wd_dslash_mrhs(b, a, g, 0, 0, -BATCH_KAPPA, None, 0.0, nr, None, dims, W.WD_F32, 12)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(n_steps):
        if k & 1:
            W.wd_dslash_mrhs(a, b, g, 1, 0, -BATCH_KAPPA, None, 0.0, nr, None, dims, W.WD_F32, 12)
        else:
            W.wd_dslash_mrhs(b, a, g, 0, 0, -BATCH_KAPPA, None, 0.0, nr, None, dims, W.WD_F32, 12)
    e1.record()
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / n_steps
    bps = 8 * 48 / nr + 96 + 96
    out["mrhs_dslash"] = {"dims": list(dims), "nrhs": nr, "prec": "f32",
                          "us_per_launch": dt * 1e6,
                          "gflops": FLOPS_PER_SITE * Vh * nr / dt / 1e9,
                          "bytes_per_rhs_site": bps,
                          "gbs": bps * Vh * nr / dt / 1e9}
    return out


NN_KAPPA = 0.1370     # the learned-preconditioner workload: beyond the critical region of these links


def nn_section(W, torch, U_big):
    """Learned gauge-covariant preconditioner at kappa = 0.137 (beyond the
    critical region of these links, where restarted GCR on D stagnates): train
    on 16^3x32 (4096 on-GPU pairs (D x, x), Adam, starting from the hopping
    series 1 + kH + k^2H^2 + k^3H^3), then time-to-1e-10 on 16^3x32 and 32^3x64
    of flexible CG on the even-odd normal equations Mhat^+ Mhat x_e =
    Mhat^+ bhat_e with the preconditioner N_e N_e^+ (N_e the even-even block of
    the network, run with BF16 activations) for the trained network, the
    untrained series and no network (plain even-odd CGNR), against plain FP64
    even-odd CG and the mixed-precision even-odd CG on the same GPU.  The
    network is local and gauge covariant, so the weights trained on the small
    lattice serve the large one.  Every time is one solve after a short
    warm-up solve; the true residual is the solver's FP64 one."""
    from synth import fields
    out = {}
    train_dims = (16, 16, 16, 32)
    U = fields.su3_links(train_dims)
    Ud = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
    p = W.wd_nn_train_params_default()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tinfo = W.wd_nn_train(w, Ud, NN_KAPPA, train_dims, p)
    torch.cuda.synchronize()
    tinfo["wall_s"] = time.perf_counter() - t0
    tinfo["samples"] = p.samples
    tinfo["batch"] = p.batch
    tinfo["dims"] = list(train_dims)
    out["training"] = tinfo
    series = torch.zeros_like(w)
    W.wd_nn_init(series, NN_KAPPA)
    for dims in (train_dims, (32, 32, 32, 64)):
        Uh = U if dims == train_dims else U_big
        Ug = torch.from_numpy(Uh.view(np.float64).reshape(-1)).cuda()
        b = torch.from_numpy(fields.gaussian_spinor(dims, seed=2026).view(np.float64)
                             .reshape(-1)).cuda()
        x = torch.zeros_like(b)
        res = {}
        for name, wts in (("fcg_trained", w), ("fcg_series", series), ("cgnr_plain", None)):
            q = W.wd_solve_params_default()
            q.maxiter = 5
            W.wd_solve_fcg(x, b, Ug, NN_KAPPA, dims, wts, q, check=False)  # warm-up
            x.zero_()
            q = W.wd_solve_params_default()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = W.wd_solve_fcg(x, b, Ug, NN_KAPPA, dims, wts, q, check=False)
            torch.cuda.synchronize()
            res[name] = {"wall_s": time.perf_counter() - t0, "iters": info["iters"],
                         "reliable_updates": info["reliable_updates"], "status": info["status"],
                         "fallback_iters": info["fallback_iters"],
                         "true_residual": info["true_residual"]}
        for name, inner in (("cg_plain_f64", W.WD_F64), ("cg_mixed_f16", W.WD_F16)):
            q = W.wd_solve_params_default()
            q.inner_prec = inner
            q.maxiter = 20
            W.wd_solve_ex(x, b, Ug, NN_KAPPA, dims, q, check=False)  # warm-up
            q.maxiter = 100000
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = W.wd_solve_ex(x, b, Ug, NN_KAPPA, dims, q, check=False)
            torch.cuda.synchronize()
            res[name] = {"wall_s": time.perf_counter() - t0, "iters": info["iters"],
                         "status": info["status"], "true_residual": info["true_residual"]}
        for name in ("fcg_trained", "fcg_series", "cgnr_plain", "cg_mixed_f16"):
            res[name]["speedup_vs_plain_f64_cg"] = (res["cg_plain_f64"]["wall_s"]
                                                    / res[name]["wall_s"])
        out["x".join(map(str, dims))] = res
        del Ug, b, x
        torch.cuda.empty_cache()
    out["config"] = {"kappa": NN_KAPPA, "network": "3 layers, 12->24->24->12 complex channels, "
                     "nearest-neighbour gauge-covariant, BF16 tensor-core contraction (tcgen05), "
                     "FP32 accumulation, BF16 activations between layers",
                     "solver": "flexible CG (Polak-Ribiere beta) on the even-odd normal equations "
                     "Mhat^+ Mhat, preconditioner N_e N_e^+ (the even-even block of the network), "
                     "FP32 vectors, FP64 reliable updates every 50 iterations; plain CG fallback",
                     "tol": 1e-10}
    return out


def profile_case(name):
    """A short fixed workload for an ncu capture (nothing timed or reported):
    ``mrhs``      4 multi-RHS hopping launches (12 right-hand sides, FP32,
                  24^3x48);
    ``solve_f32`` / ``solve_f16``  2 mixed-precision CG solves to 1e-10 on
                  24^3x48 (kappa 0.137);
    ``batch``     one batched FP32-inner solve of 12 point sources on 24^3x48
                  (one launch per step);
    ``batch_persistent``  the same with one persistent launch per iteration;
    ``nn_bf16``   2 applications of the series network with BF16 activations
                  on 24^3x48;
    ``fcg``       one learned-preconditioner solve (series weights, flexible CG
                  on the even-odd system) on 16^3x32 at kappa 0.137;
    ``train``     4 Adam steps of 16 samples on 16^3x32 (forward, adjoint and
                  tensor-core weight-gradient kernels);
    ``nn``        2 applications of the series-initialised network (three
                  tensor-core layers) on 16^3x32;
    ``staged``    4 FP16 parity dslashes on 32^3x64 with the far neighbours
                  staged by bulk copies (WD_STAGE_NEIGHBOURS), then 4 with the
                  unstaged kernel (128-site CTAs forced, so no tuning runs)."""
    import torch
    from synth import fields
    import paper_0810_5365_gb300 as W
    torch.cuda.set_device(0)
    if name == "mrhs":
        dims, nr = (24, 24, 24, 48), 12
        Vh = int(np.prod(dims)) // 2
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        g = W.alloc_gauge(dims, W.WD_F32, 12)
        W.wd_pack_gauge(g, Ud, dims, W.WD_F32, 12)
        h = W.wd_spinor_bytes(dims, 0, W.WD_F32)
        a = torch.zeros(nr * h, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        src = torch.from_numpy(fields.gaussian_spinor(dims, nsites=Vh).view(np.float64)
                               .reshape(-1)).cuda()
        for r in range(nr):
            W.wd_pack_spinor(a[r * h:(r + 1) * h], src, dims, 1, W.WD_F32)
        for _ in range(4):
            W.wd_dslash_mrhs(b, a, g, 0, 0, -BATCH_KAPPA, None, 0.0, nr, None, dims, W.WD_F32, 12)
    elif name == "staged":
        dims = DIMS
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        g = W.alloc_gauge(dims, W.WD_F16, 12)
        W.wd_pack_gauge(g, Ud, dims, W.WD_F16, 12)
        del Ud
        src = torch.from_numpy(fields.gaussian_spinor(dims).view(np.float64).reshape(-1)).cuda()
        a = W.alloc_spinor(dims, W.WD_FULL, W.WD_F16)
        W.wd_pack_spinor(a, src, dims, W.WD_FULL, W.WD_F16)
        del src
        h = W.wd_spinor_bytes(dims, W.WD_EVEN, W.WD_F16)
        W.wd_dslash_set_block(128)
        for recon in (12 | W.WD_STAGE_NEIGHBOURS, 12):
            for _ in range(4):
                W.wd_dslash_ex(a[:h], a[h:], g, W.WD_EVEN, 0, -KAPPA, None, 0.0, None, 0.0,
                               None, dims, W.WD_F16, recon)
        W.wd_dslash_set_block(0)
    elif name in ("solve_f32", "solve_f16"):
        dims = SOLVE_DIMS
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        bd = torch.from_numpy(fields.gaussian_spinor(dims, seed=2025).view(np.float64)
                              .reshape(-1)).cuda()
        x = torch.zeros_like(bd)
        p = W.wd_solve_params_default()
        p.inner_prec = W.WD_F32 if name == "solve_f32" else W.WD_F16
        for _ in range(2):
            x.zero_()
            W.wd_solve_ex(x, bd, Ud, SOLVE_KAPPA, dims, p)
    elif name == "batch":
        dims = (24, 24, 24, 48)
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        bs = [fields.point_source(dims, 0, r // 3, r % 3) for r in range(12)]
        b = torch.from_numpy(np.ascontiguousarray(np.stack(bs)).view(np.float64)).cuda()
        probs = [{"dims": dims, "kappa": BATCH_KAPPA, "nrhs": 12, "gauge": Ud, "b": b,
                  "x": torch.zeros_like(b)}]
        p = W.wd_solve_params_default()
        p.inner_prec = W.WD_F32
        W.wd_solve_batch(probs, p)
    elif name == "batch_persistent":
        # the same solve with one persistent launch per iteration
        dims = (24, 24, 24, 48)
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        bs = [fields.point_source(dims, 0, r // 3, r % 3) for r in range(12)]
        b = torch.from_numpy(np.ascontiguousarray(np.stack(bs)).view(np.float64)).cuda()
        probs = [{"dims": dims, "kappa": BATCH_KAPPA, "nrhs": 12, "gauge": Ud, "b": b,
                  "x": torch.zeros_like(b)}]
        p = W.wd_solve_params_default()
        p.inner_prec = W.WD_F32
        W.wd_set_batch_mode(1)
        W.wd_solve_batch(probs, p)
    elif name == "fcg":
        # one learned-preconditioner solve (series weights) on 16^3x32 at
        # kappa = 0.137: flexible CG on the even-odd system with N_e N_e^+
        dims = (16, 16, 16, 32)
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        b = torch.from_numpy(fields.gaussian_spinor(dims, seed=2026).view(np.float64)
                             .reshape(-1)).cuda()
        x = torch.zeros_like(b)
        w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
        W.wd_nn_init(w, NN_KAPPA)
        W.wd_solve_fcg(x, b, Ud, NN_KAPPA, dims, w)
    elif name == "train":
        dims = (16, 16, 16, 32)
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
        p = W.wd_nn_train_params_default()
        p.samples = 64
        W.wd_nn_train(w, Ud, NN_KAPPA, dims, p)
    elif name == "nn":
        dims = (16, 16, 16, 32)
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        g = W.alloc_gauge(dims, W.WD_F32, 12)
        W.wd_pack_gauge(g, Ud, dims, W.WD_F32, 12)
        w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
        W.wd_nn_init(w, NN_KAPPA)
        src = torch.from_numpy(fields.gaussian_spinor(dims).view(np.float64).reshape(-1)).cuda()
        a = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
        W.wd_pack_spinor(a, src, dims, W.WD_FULL, W.WD_F32)
        b = torch.zeros_like(a)
        for _ in range(2):
            W.wd_nn_apply(b, a, w, g, dims)
    elif name == "nn_bf16":
        # two applications of the series network with BF16 activations on
        # 24^3x48 (links 127 MB: the working set exceeds L2)
        dims = (24, 24, 24, 48)
        Ud = torch.from_numpy(fields.su3_links(dims).view(np.float64).reshape(-1)).cuda()
        g = W.alloc_gauge(dims, W.WD_F32, 12)
        W.wd_pack_gauge(g, Ud, dims, W.WD_F32, 12)
        w = torch.zeros(W.WD_NN_PARAMS, dtype=torch.float32, device="cuda")
        W.wd_nn_init(w, NN_KAPPA)
        src = torch.from_numpy(fields.gaussian_spinor(dims).view(np.float64).reshape(-1)).cuda()
        a = W.alloc_spinor(dims, W.WD_FULL, W.WD_F32)
        W.wd_pack_spinor(a, src, dims, W.WD_FULL, W.WD_F32)
        b = torch.zeros_like(a)
        for _ in range(2):
            W.wd_nn_apply_ex(b, a, w, g, dims, W.WD_NN_BF16)
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    print(json.dumps({"profile": name, "ok": True}), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_0810_5365_gb300 as W
    W.wd.lib()
    stream = torch.cuda.current_stream()
    W.wd_set_stream(stream)

    dims = DIMS
    Vh = int(np.prod(dims)) // 2
    U, psi = make_fields(dims)
    Ud = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    from synth import fields
    src = fields.to_half(psi, dims, 1)
    srcd = torch.from_numpy(src.view(np.float64).reshape(-1)).cuda()

    results = {}
    peaks, peak_kind = measured_peaks()
    gauges = {}
    variants = [("f32", W.WD_F32, 12, args.steps), ("f16", W.WD_F16, 12, args.steps),
                ("f64", W.WD_F64, 18, max(1, args.steps // 8)),
                ("f32_tg", W.WD_F32, 12 | W.WD_TEMPORAL_GAUGE, args.steps),
                ("f16_tg", W.WD_F16, 12 | W.WD_TEMPORAL_GAUGE, args.steps),
                ("f16_staged", W.WD_F16, 12 | W.WD_STAGE_NEIGHBOURS, args.steps)]
    if args.quick:
        variants = variants[:1]
    Utg = None
    with ClockSampler(local) as clk:
        for name, pid, recon, steps in variants:
            src_links = Ud
            if recon & W.WD_TEMPORAL_GAUGE:
                if Utg is None:
                    # the paper's gauge-fixing trick: temporal gauge on the device
                    Utg = torch.empty_like(Ud)
                    om = torch.empty(int(np.prod(dims)) * 18, dtype=torch.float64, device="cuda")
                    W.wd_gauge_fix_temporal(Utg, om, Ud, dims)
                    del om
                src_links = Utg
            g = W.alloc_gauge(dims, pid, recon & 0xFF)
            W.wd_pack_gauge(g, src_links, dims, pid, recon & 0xFF)
            a = W.alloc_spinor(dims, W.WD_ODD, pid)
            b = W.alloc_spinor(dims, W.WD_EVEN, pid)
            W.wd_pack_spinor(a, srcd, dims, W.WD_ODD, pid)
            W.wd_pack_spinor(b, srcd, dims, W.WD_EVEN, pid)
            if name == "f32":
                gauges[name] = (g, a, b, pid)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            dt = time_dslash(W, torch, pid, recon, g, (a, b), dims, steps, args.warmup, stream)
            if world > 1:
                dt = max_over_ranks(dt, "cuda")
            results[name] = (dt, steps)
            del g, a, b
        # the headline launches once more, captured as one CUDA graph
        g32, a32, b32, _ = gauges["f32"]
        dt_graph = time_dslash_graph(W, torch, g32, (a32, b32), dims, args.steps)
        # the paper's Fig. 1 operator: Mhat = 1 - kappa^2 D_eo D_oe on the even
        # sites (two parity dslashes, the second with the fused epilogue)
        tmp_o = W.alloc_spinor(dims, W.WD_ODD, W.WD_F32)
        out_e = W.alloc_spinor(dims, W.WD_EVEN, W.WD_F32)
        n_mhat = max(1, args.steps // 2)
        for _ in range(args.warmup):
            W.wd_mhat(out_e, b32, g32, tmp_o, KAPPA, 0, dims, W.WD_F32)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_mhat):
            W.wd_mhat(out_e, b32, g32, tmp_o, KAPPA, 0, dims, W.WD_F32)
        e1.record(stream)
        e1.synchronize()
        dt_mhat = e0.elapsed_time(e1) / 1e3
        del tmp_o, out_e
        # end to end through the C ABI with pinned host buffers: every step
        # copies its input spinor in, applies the operator and copies the
        # result out.  Three streams and two device buffer pairs let step
        # k+1's input copy and step k-1's output copy run under step k's
        # kernel (the host link carries both directions at once); every copy
        # is inside the timed region.
        g, a, b, pid = gauges["f32"]
        nb = W.wd_spinor_bytes(dims, W.WD_ODD, W.WD_F32)
        h_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        h_out = [torch.empty(nb, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        h_in.copy_(a)
        a2, b2 = [a, torch.empty_like(a)], [b, torch.empty_like(b)]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        k_e2e = max(1, min(args.steps, 50))

        def e2e_run(k, e_first=None, e_last=None):
            ev_cmp = [torch.cuda.Event() for _ in range(k)]
            ev_in = [torch.cuda.Event() for _ in range(k)]
            ev_out = [torch.cuda.Event() for _ in range(k)]
            if e_first is not None:
                e_first.record(s_in)
            W.wd_set_stream(s_cmp)
            for i in range(k):
                j = i & 1
                if i >= 2:
                    s_in.wait_event(ev_cmp[i - 2])    # a2[j] consumed
                with torch.cuda.stream(s_in):
                    a2[j].copy_(h_in, non_blocking=True)
                ev_in[i].record(s_in)
                s_cmp.wait_event(ev_in[i])
                if i >= 2:
                    s_cmp.wait_event(ev_out[i - 2])   # b2[j] copied out
                W.wd_dslash(b2[j], a2[j], g, KAPPA, W.WD_EVEN, dims, W.WD_F32)
                ev_cmp[i].record(s_cmp)
                s_out.wait_event(ev_cmp[i])
                with torch.cuda.stream(s_out):
                    h_out[j].copy_(b2[j], non_blocking=True)
                ev_out[i].record(s_out)
            if e_last is not None:
                e_last.record(s_out)
            W.wd_set_stream(stream)

        e2e_run(3)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2e_run(k_e2e, e0, e1)
        e1.synchronize()
        torch.cuda.synchronize()
        dt_e2e = e0.elapsed_time(e1) / 1e3
        # the result of the last step reached the host intact
        assert torch.equal(h_out[(k_e2e - 1) & 1], b2[(k_e2e - 1) & 1].cpu())
        del a2, b2
    clocks = clk.summary()
    del gauges, g, a, b, Ud, srcd
    torch.cuda.empty_cache()

    dt, steps = results["f32"]
    gflops = replica_value(FLOPS_PER_SITE * Vh * steps, world, dt) / 1e9
    launch_s = dt / steps
    achieved = BYTES_PER_SITE["f32"] * Vh / launch_s / 1e9
    line = {
        "metric": METRIC, "value": gflops, "unit": "Gflops", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": DATA,
        "config": headline_config(dims, world),
        "dslash_gbs": achieved,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": profiled_traffic("f32"),
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                     "bytes_per_site": BYTES_PER_SITE["f32"],
                     "frac_of_nominal_8tbs": achieved / 8000.0},
        "mhat": {"ms_per_step": 1e3 * dt_mhat / n_mhat,
                 "value": (2 * FLOPS_PER_SITE + 48) * Vh * n_mhat * world / dt_mhat / 1e9,
                 "unit": "Gflops", "steps": n_mhat,
                 "note": "even-odd operator 1 - kappa^2 D_eo D_oe (the paper's Fig. 1), FP32, "
                         "12-real links, 2 x 1320 + 48 flops per even site"},
        "graph": {"ms_per_step": 1e3 * dt_graph / args.steps,
                  "value": FLOPS_PER_SITE * Vh * args.steps * world / dt_graph / 1e9,
                  "unit": "Gflops", "note": "the same launches captured as one CUDA graph"},
        "gpu_launches": steps,
        "paper_context": {"tesla_c870_gflops": 68, "gtx280_gflops": 92,
                          "note": "the paper's FP32 Wilson-Dirac operator on G80/GT200 cards, "
                                  "lattice volume not stated: context, not the same workload"},
        "variants": {},
    }
    for name in ("f16", "f64", "f32_tg", "f16_tg", "f16_staged"):
        if name not in results:
            continue
        d, st = results[name]
        if name == "f16_staged":
            bps = BYTES_PER_SITE["f16"]
        else:
            bps = BYTES_PER_SITE[name] if name in BYTES_PER_SITE else tg_bytes_per_site(name, dims)
        ach = bps * Vh / (d / st) / 1e9
        line["variants"][name] = {
            "value": FLOPS_PER_SITE * Vh * st * world / d / 1e9, "unit": "Gflops",
            "steps": st, "ms_per_step": 1e3 * d / st, "dslash_gbs": ach,
            "frac": ach / peaks["hbm_gbs"], "bytes_per_site": bps,
            "recon": 18 if name == "f64" else 12, "traffic": profiled_traffic(name)}
        if name.endswith("_tg"):
            line["variants"][name]["note"] = (
                "temporal gauge: U_t = 1 off the last time slice (not loaded); effective "
                "Gflops still count the nominal 1320 flops/site")
        if name == "f16_staged":
            line["variants"][name]["note"] = (
                "FP16 with the +-z and +-t neighbour spinors staged in shared memory by "
                "bulk asynchronous (TMA) copies, one mbarrier per warp; bit-identical to f16, "
                "and the kernel the CTA-size tuner chooses for plain FP16 calls on this lattice")
        line["gpu_launches"] += st
    line["e2e"] = {"value": FLOPS_PER_SITE * Vh * k_e2e * world / dt_e2e / 1e9, "unit": "Gflops",
                   "steps": k_e2e, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
                   "overlap": "3 streams, 2 device buffer pairs: step k+1's input copy and "
                              "step k-1's output copy run under step k's kernel"}
    line["gpu_launches"] += k_e2e + args.steps + 2 * n_mhat  # e2e, graph replay, Mhat
    line["clocks"] = clocks
    if not args.no_solve and not args.quick:
        line["solve"] = solve_section(W, torch)
        torch.cuda.empty_cache()
        line["batch"] = batch_section(W, torch)
        torch.cuda.empty_cache()
        line["learned_preconditioner"] = nn_section(W, torch, U)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(U, psi, dims)
        if "solve" in line and not args.no_oracle_cg:
            # the oracle's plain FP64 CG to 1e-10 on the solve problem, timed
            # whole (about 100 s on 16 host cores), beside the GPU's solves
            oc = oracle_cg_full()
            oc["gpu_plain_f64_cg_s"] = line["solve"]["f64"]["wall_s"]
            oc["gpu_mixed_f16_cg_s"] = line["solve"]["f16"]["wall_s"]
            oc["gpu_plain_f64_speedup"] = oc["wall_s"] / oc["gpu_plain_f64_cg_s"]
            oc["gpu_mixed_f16_speedup"] = oc["wall_s"] / oc["gpu_mixed_f16_cg_s"]
            line["cpu_baseline"]["oracle_cg_24x24x24x48"] = oc
    if rank == 0:
        # the compact summary right after the config, ahead of the long sections
        head = {}
        for k, v in line.items():
            head[k] = v
            if k == "config":
                head["summary"] = compact_summary(line)
        line = head
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--quick", action="store_true", help="FP32 dslash only")
    ap.add_argument("--no-solve", action="store_true", help="skip the 24^3x48 solver comparison")
    ap.add_argument("--no-oracle-cg", action="store_true",
                    help="skip the oracle's full FP64 CG timing (about 100 s of host time)")
    ap.add_argument("--profile", choices=["mrhs", "solve_f32", "solve_f16", "batch",
                                          "batch_persistent", "fcg", "train", "nn", "nn_bf16",
                                          "staged"],
                    help="run a short fixed workload for an ncu capture and exit")
    args = ap.parse_args()
    if args.profile:
        return profile_case(args.profile)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
