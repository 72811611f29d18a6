/*
 * wd.h -- C ABI of libwd, a GB300 (sm_103a) library for the Wilson-Dirac
 * operator and the Krylov solve that calls it.
 *
 * Paper: K. Barros, R. Babich, R. Brower, M. A. Clark, C. Rebbi, "Blasting
 * through lattice calculations using CUDA", Lattice 2008 (arXiv:0810.5365).
 * The paper implements a CUDA kernel "Dslash" (the Wilson-Dirac hopping term
 * restricted to the even or odd sub-lattice, with its adjoint) and an
 * even-odd preconditioned conjugate-gradient solver built from it, a
 * double-precision dot product and BLAS-like vector kernels (section
 * "Wilson inverter: Main features"); its Fig. 1 benchmarks the preconditioned
 * operator 1 - kappa^2 D_eo D_oe.  The operator itself is not printed there;
 * this library uses the standard Wilson fermion (r = 1, hopping-parameter
 * normalisation):
 *
 *   D psi(x) = psi(x) - kappa * H psi(x),
 *   H psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                     + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu) ],
 *
 * chiral gamma basis (gamma_5 = diag(1,1,-1,-1)), periodic boundaries in x, y,
 * z and antiperiodic ones in t.  H^+ exchanges the two projectors.
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every call
 * ---------------------------------------------------------------------------
 * dims[4]   lattice extents L0 (x), L1 (y), L2 (z), L3 (t).  Every extent must
 *           be even and >= 2 (else WD_ERR_DIMS); V = L0 L1 L2 L3, Vh = V/2.
 * parity    of site x is (x0+x1+x2+x3) & 1; WD_EVEN = 0, WD_ODD = 1.
 *           WD_FULL (-1) means both parities (even half first, then odd).
 * canonical FP64 layouts (row-major complex double, re then im):
 *           full spinor   [V][4 spin][3 colour]
 *           half spinor   [Vh][4][3]: the sites of one parity in increasing
 *                         lexicographic order (site i sits at i >> 1)
 *           gauge         [4 mu][V][3 row][3 col]; U_mu(x) links x -> x+mu
 *           lexicographic site i = x0 + L0*(x1 + L1*(x2 + L2*x3)).
 * packed    formats are opaque device buffers produced by wd_pack_* and sized
 *           by wd_spinor_bytes / wd_gauge_bytes (site-blocked structure of
 *           arrays: blocks of 32 checkerboard sites, each block holding one
 *           128-bit vector per site per component group).  Precisions:
 *           WD_F64 (double), WD_F32 (float), WD_F16 (half with one float
 *           scale per site for spinors; plain half for SU(3) links).  Links
 *           are stored with 18 reals (recon = 18) or as their first two rows,
 *           12 reals (recon = 12), the third row being rebuilt in registers
 *           as conj(row0 x row1) (paper, section "Performance": only two
 *           columns of each gauge matrix are read; rows are used here, which
 *           is equivalent for SU(3)).  WD_F16 links support recon = 12 only.
 * pointers  unless stated otherwise, buffer arguments are DEVICE pointers,
 *           16-byte aligned (else WD_ERR_ALIGN), owned by the caller; the
 *           library never frees them.  Calls are asynchronous on the stream
 *           set by wd_set_stream (default: the legacy default stream), except
 *           wd_solve / wd_solve_ex, which return after the solve.
 * errors    every int-returning call returns a WD_* status; no C++ exception
 *           crosses this interface.  WD_ERR_CUDA means a CUDA runtime call
 *           failed (wd_last_cuda_error gives its code).  The library is not
 *           thread-safe: use it from one host thread at a time.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { WD_F64 = 0, WD_F32 = 1, WD_F16 = 2 };

/* OR into a `recon` argument (12 | WD_TEMPORAL_GAUGE, ...) when the packed
 * gauge field is in temporal gauge (see wd_gauge_fix_temporal): the hopping
 * kernels then treat U_t(x) as the identity on every slice but t = L3-1 and
 * neither load nor apply it. */
enum { WD_TEMPORAL_GAUGE = 0x100 };

/* OR into the `recon` argument of wd_dslash_ex: FP16 hopping in which each
 * warp stages the spinors of its +-z and +-t neighbours (four whole 32-site
 * blocks of the other parity) in shared memory with bulk asynchronous copies
 * (the TMA engine) while it computes its x and y hops.  Results are
 * bit-identical to the unstaged kernel.  Requires prec = WD_F16, recon = 12,
 * no temporal gauge, norm2 == NULL and L0*L1/2 a multiple of 32; WD_ERR_ARG
 * otherwise.  Without this bit the CTA-size tuner (wd_dslash_set_block) may
 * choose the same kernel for such calls when it is the faster one.  The wait
 * for the copies is bounded (wd_set_wait_limit); should
 * it give up, the kernel writes NaN to the sites of that warp (so any later
 * norm, solve or check of the output fails) instead of hanging, and raises
 * the device's fault flag, which wd_async_status reports. */
enum { WD_STAGE_NEIGHBOURS = 0x200 };
enum { WD_EVEN = 0, WD_ODD = 1, WD_FULL = -1 };

enum {
    WD_OK = 0,
    WD_ERR_NULL = 1,       /* a required pointer is NULL */
    WD_ERR_DIMS = 2,       /* an extent is odd, < 2, or the volume overflows */
    WD_ERR_PREC = 3,       /* unknown precision / unsupported (prec, recon) */
    WD_ERR_ALIGN = 4,      /* a device buffer is not 16-byte aligned */
    WD_ERR_ALIAS = 5,      /* output aliases an input that is read at neighbours */
    WD_ERR_NOCONV = 6,     /* solver hit maxiter; x holds the best iterate */
    WD_ERR_NONFINITE = 7,  /* NaN/Inf met in a residual norm */
    WD_ERR_TIMEOUT = 8,    /* a bounded device-side wait gave up */
    WD_ERR_CUDA = 9,       /* a CUDA runtime call failed */
    WD_ERR_ARG = 10,       /* another argument is out of range */
    WD_ERR_BREAKDOWN = 11, /* Krylov breakdown (p^+ A p <= 0) */
    WD_ERR_SCRATCH = 12    /* lattice too large for wd_dslash_ex_noalloc's fixed scratch */
};

/* ------------------------------------------------------------------ */
/* state                                                               */
/* ------------------------------------------------------------------ */

/* Stream for all following calls (a cudaStream_t; NULL = legacy default). */
int wd_set_stream(void *cuda_stream);
void *wd_get_stream(void);

/* Human-readable name of a status code (static string, never NULL). */
const char *wd_error_string(int status);

/* cudaError_t of the last failed CUDA call (0 if none). */
int wd_last_cuda_error(void);

/* Free the library's cached workspace (solver fields, reduction scratch,
 * captured graphs).  Caller buffers are untouched.  Safe to call twice. */
void wd_finalize(void);

/* ------------------------------------------------------------------ */
/* layout: sizes, pack, unpack (paper, section "Data layout")          */
/* ------------------------------------------------------------------ */

/* Bytes of a packed spinor field of one parity (or both, parity = WD_FULL);
 * 0 on invalid arguments. */
size_t wd_spinor_bytes(const int dims[4], int parity, int prec);

/* Bytes of a packed gauge field (all 4 directions, both parities); 0 on
 * invalid arguments (e.g. WD_F16 with recon 18). */
size_t wd_gauge_bytes(const int dims[4], int prec, int recon);

/* Canonical FP64 gauge field (device) -> packed gauge of (prec, recon),
 * split by parity of the link's base site. */
int wd_pack_gauge(void *dst, const double *src_canonical, const int dims[4],
                  int prec, int recon);

/* Canonical FP64 spinor (device; half layout for parity 0/1, full layout for
 * WD_FULL) -> packed spinor of prec. */
int wd_pack_spinor(void *dst, const double *src_canonical, const int dims[4],
                   int parity, int prec);

/* Packed spinor -> canonical FP64 (device), inverse of wd_pack_spinor. */
int wd_unpack_spinor(double *dst_canonical, const void *src, const int dims[4],
                     int parity, int prec);

/* Packed spinor of src_prec -> packed spinor of dst_prec (same parity). */
int wd_convert_spinor(void *dst, int dst_prec, const void *src, int src_prec,
                      const int dims[4], int parity);

/* ------------------------------------------------------------------ */
/* the hopping operator (paper, section "Wilson inverter")             */
/* ------------------------------------------------------------------ */

/*
 * wd_dslash: parity p in {WD_EVEN, WD_ODD}:
 *     out_p = -kappa * H_{p,1-p} in_{1-p}
 * (in is the packed half field of the opposite parity, out of parity p);
 * parity WD_FULL:
 *     out = in - kappa * H in = D in    (packed full fields).
 * gauge is packed with the same prec and recon 12 (use wd_dslash_ex for
 * recon 18).  out must not alias in (WD_ERR_ALIAS).
 */
int wd_dslash(void *out, const void *in, const void *gauge, double kappa,
              int parity, const int dims[4], int prec);

/* Same with H^+ (projectors exchanged): D^+ = gamma_5 D gamma_5. */
int wd_dslash_dag(void *out, const void *in, const void *gauge, double kappa,
                  int parity, const int dims[4], int prec);

/*
 * General parity-restricted hopping application with a fused epilogue:
 *     out_p = a * H_{p,1-p} in_{1-p}  [+ bx * x_p]  [+ cy * y_p]
 * (H^+ when dagger != 0).  x and y may be NULL (term dropped) and may alias
 * out; in must not.  If norm2 != NULL (device double*), ||out_p||^2 is
 * written there: summed in the working precision (FP64 for WD_F64, else FP32)
 * over each 128-site CTA, then over the CTA partials in FP64 in a fixed order
 * by a second, one-CTA launch on the same stream (deterministic).  recon is
 * 12 or 18.
 */
int wd_dslash_ex(void *out, const void *in, const void *gauge, int parity, int dagger,
                 double a, const void *x, double bx, const void *y, double cy,
                 double *norm2, const int dims[4], int prec, int recon);

/*
 * wd_dslash_ex_noalloc: wd_dslash_ex (same arguments, same results) for
 * callers that cannot let the library allocate device memory.  The paper has
 * no counterpart; this is an interface addition.  recon takes the same flag
 * bits as in wd_dslash_ex (| WD_TEMPORAL_GAUGE, | WD_STAGE_NEIGHBOURS, with
 * the same restrictions); the staged kernel reduces nothing and so uses no
 * scratch at all.
 *
 * Who needs it: code that records its launches into a CUDA graph by stream
 * capture (allocating during a capture is not allowed), applications whose
 * device memory is owned by another allocator (e.g. a framework's caching
 * allocator that has reserved the GPU), and latency-critical loops that must
 * not hit the device-wide synchronisation of cudaMalloc/cudaFree.
 * wd_dslash_ex may allocate its reduction scratch on first use or when a
 * larger lattice needs more; this variant never calls cudaMalloc, cudaFree or
 * any allocating routine.
 *
 * Its reduction scratch is a fixed array compiled into libwd (16384 FP64
 * partial sums, 128 KB), held by every GPU that loads the library until the
 * process exits.  Limit: V/2 <= 2,097,152 sites
 * (16384 CTAs of 128 sites); larger lattices return WD_ERR_SCRATCH before
 * any work is queued.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array: with
 * norm2 != NULL the hopping kernel leaves one partial sum per CTA there and a
 * second, one-CTA launch on the same stream adds them into *norm2.  Calls
 * that overlap on the GPU (several streams, or several host threads) race on
 * the array.
 */
int wd_dslash_ex_noalloc(void *out, const void *in, const void *gauge, int parity,
                         int dagger, double a, const void *x, double bx, const void *y,
                         double cy, double *norm2, const int dims[4], int prec, int recon);

/*
 * Even-odd preconditioned operator on the even sub-lattice (paper Fig. 1):
 *     out_e = (1 - kappa^2 H_eo H_oe) in_e          (dagger = 0)
 *     out_e = (1 - kappa^2 H^+_eo H^+_oe) in_e      (dagger = 1, its adjoint)
 * tmp is a caller-owned packed odd half field of the same prec.
 */
int wd_mhat(void *out, const void *in, const void *gauge, void *tmp, double kappa,
            int dagger, const int dims[4], int prec, int recon);

/*
 * Multi-right-hand-side hopping application (batched form of wd_dslash_ex):
 * nrhs packed half fields laid out back to back (consecutive fields
 * wd_spinor_bytes(dims, parity, prec) apart) share one gauge field:
 *     out_r = a * H_{p,1-p} in_r  [+ bx * x_r]          r = 0 .. nrhs-1
 * (H^+ when dagger != 0).  The CTAs that cover the right-hand sides of the
 * same sites run together, so each link comes from memory once per site and
 * serves every right-hand side from cache.  The tile shape (right-hand-side
 * warps per CTA, right-hand sides per thread) comes from the autotuner
 * below.  x may be NULL or alias out;
 * in must not.  If norm2 != NULL (device, nrhs doubles) it receives
 * ||out_r||^2, summed in a fixed order (in the working precision over each
 * warp's 32 sites, then in FP64).  1 <= nrhs <= 32.
 */
int wd_dslash_mrhs(void *out, const void *in, const void *gauge, int parity, int dagger,
                   double a, const void *x, double bx, int nrhs, double *norm2,
                   const int dims[4], int prec, int recon);

/*
 * Autotuner of the multi-right-hand-side tile shape of wd_dslash_mrhs and of
 * the hopping launches of wd_solve_batch, and of the CTA size of the
 * single-field hopping kernel (wd_dslash_set_block below); the paper has no
 * such component.
 * A shape code is w (1, 2, 4 or 8 right-hand-side warps per CTA, one
 * right-hand side per thread) or, for FP32 only, 16 + w (w = 1, 2 or 4 warps,
 * two right-hand sides per thread: each link is loaded and rebuilt once for
 * both).  Every shape gives bit-identical results.
 *
 * enable = 1 (the default): a batch shape (precision, link format, dagger,
 * fused norm, tile count, largest nrhs, problem count) met for the first time
 * outside stream capture is timed with every tile shape (CUDA events, one
 * warm-up and three launches each) on temporary output buffers, so no caller
 * data is written; the fastest shape is used from then on.  Tuning needs
 * device memory for one copy of the outputs; without it the default shape (4)
 * is kept.  wd_solve_batch tunes its inner launches before it captures its
 * iteration graph.  enable = 0: shapes not yet tuned use the default.
 * Returns the previous setting.
 */
int wd_set_autotune(int enable);

/* Force the CTA size (64, 128 or 256 sites) of every single-field hopping
 * launch without a fused reduction, or go back to the tuned sizes (sites =
 * 0).  The autotuner (wd_set_autotune) times the three sizes for each new
 * (link format, dagger, temporal gauge, lattice extents) met outside stream
 * capture, on a temporary output, and keeps the fastest; for FP16 with
 * 12-real links (no temporal gauge) on lattices whose (z, t) slices hold a
 * multiple of 32 sites of one parity it also times the kernel that stages
 * the far neighbours in shared memory (see WD_STAGE_NEIGHBOURS, whose
 * bounded wait and wd_async_status then apply).  Every candidate gives
 * bit-identical fields.  Launches with a fused norm keep 128 sites, so that
 * the summation order of the norm never depends on a timing.
 * wd_dslash_ex_noalloc never tunes (it would allocate) but uses a choice
 * already made.  A forced size always runs the unstaged kernel.  WD_ERR_ARG
 * for other sizes. */
int wd_dslash_set_block(int sites);

/* Launch overlap of consecutive single-field hopping kernels (the paper has
 * no such component).  enable = 1 (the default): every hopping launch of
 * wd_dslash, wd_dslash_dag, wd_dslash_ex, wd_mhat and the solvers, the
 * one-CTA launch that sums a fused norm's per-CTA partials, and the CG and
 * BiCGstab vector updates of wd_solve_ex are programmatic dependent
 * launches.  The kernel first lets the next kernel of
 * the stream be scheduled once all of its own CTAs have started, then waits
 * until the previous kernel of the stream has completed and its writes are
 * visible, before it reads or writes any memory.  So consecutive launches
 * overlap only their scheduling (the next grid's CTAs take the SM slots that
 * the last wave frees), never their memory accesses, and results are
 * bit-identical with either setting.  enable = 0: plain stream-ordered
 * launches.  Returns the previous setting. */
int wd_set_launch_overlap(int enable);

/* Force one tile shape for every multi-RHS launch (lanes = a shape code:
 * 1, 2, 4, 8, 17, 18 or 20; FP64 and FP16 launches run 16 + w as w), or go
 * back to the tuned/default shapes (lanes = 0).  WD_ERR_ARG otherwise. */
int wd_mrhs_set_lanes(int lanes);

/* Text table of the tuned shapes, one line per multi-RHS batch shape and
 * per single-field hopping shape, with the microseconds of every candidate
 * and the choice.  Writes at most len bytes,
 * NUL-terminated, into buf (buf may be NULL when len is 0).  Returns the
 * number of tuned shapes. */
int wd_tune_report(char *buf, size_t len);

/*
 * Temporal gauge (paper, section "Performance": fixing the temporal links to
 * the identity on all but one time slice saves their bandwidth, about 10 %).
 * From the canonical FP64 gauge field U_in (device) compute, on the device,
 *     omega(x, 0) = 1,  omega(x, t+1) = omega(x, t) U_t(x, t),
 *     U_out_mu(x) = omega(x) U_mu(x) omega(x+mu)^+ ,
 * so that U_out_t(x) = 1 exactly for t < L3-1.  omega_out: canonical
 * [V][3][3].  Pack U_out and pass recon | WD_TEMPORAL_GAUGE to the hopping
 * calls.  D[U_out] = omega D[U] omega^+ (gauge covariance).
 * U_out must not alias U_in.
 */
int wd_gauge_fix_temporal(double *U_out, double *omega_out, const double *U_in,
                          const int dims[4]);

/* out(x) = omega(x) in(x) (dagger = 0) or omega(x)^+ in(x) (dagger = 1);
 * canonical FP64 full spinors on the device; out may alias in. */
int wd_rotate_spinor(double *out, const double *in, const double *omega, const int dims[4],
                     int dagger);

/* ------------------------------------------------------------------ */
/* BLAS-like kernels and FP64 reductions (paper: dot product by        */
/* parallel reduction in double precision; "BLAS-like" vector kernels) */
/* ------------------------------------------------------------------ */

/* result[0] = ||x||^2 (device double*), FP64 accumulation. */
int wd_norm2(double *result, const void *x, const int dims[4], int parity, int prec);

/* result[0..1] = <x, y> = sum conj(x) y (re, im), FP64 accumulation. */
int wd_cdot(double *result, const void *x, const void *y, const int dims[4],
            int parity, int prec);

/* y = a x + b y (real a, b), elementwise in the storage precision's
 * arithmetic (FP32 for WD_F16).  With b == 0, y is output only and is not
 * read (BLAS convention), so it may be uninitialised. */
int wd_axpby(double a, const void *x, double b, void *y, const int dims[4],
             int parity, int prec);

/* ------------------------------------------------------------------ */
/* tensor cores                                                        */
/* ------------------------------------------------------------------ */

/*
 * D = A B on the 5th-generation tensor cores (tcgen05.mma, BF16 operands,
 * FP32 accumulation in tensor memory): A [M][K] and B [K][N] row-major BF16,
 * D [M][N] row-major FP32, all device memory.  M % 128 == 0, K % 16 == 0 with
 * K <= 256, N % 16 == 0 with 16 <= N <= 256 (else WD_ERR_ARG).  The paper has
 * no tensor cores; this is the contraction core of the learned preconditioner
 * below, exposed so it can be checked on its own.  Synchronous: returns
 * WD_ERR_TIMEOUT if a bounded device wait gave up.
 */
int wd_tc_gemm_bf16(float *D, const void *A, const void *B, int M, int K, int N);

/*
 * Failure-path check of the bounded device waits (no counterpart in the
 * paper).  Every spin-wait in the library's kernels (the tensor-core kernels'
 * mbarrier waits) polls at most a fixed number of times; when the polls run
 * out the kernel raises a device flag, frees what it holds and returns, and
 * the call reports WD_ERR_TIMEOUT with the context still usable.  This entry
 * point runs that path on purpose: one warp waits, through the same bounded
 * helper, on an mbarrier that nothing ever completes, for at most `spins`
 * polls (1 <= spins <= 2^24, about 100 ns each).  It returns WD_ERR_TIMEOUT
 * (the expected answer), WD_ERR_ARG for spins out of range.  Synchronous.
 */
int wd_wait_selftest(long long spins);

/*
 * Bounded waits of the asynchronous kernels (no counterpart in the paper).
 * The staged hopping kernel (WD_STAGE_NEIGHBOURS) waits for its bulk copies
 * at most `polls` times (about 100 ns each; default 2^22) before it gives
 * up, poisons its sites with NaN and raises the device's fault flag; each
 * grid-barrier wait of the persistent batched iteration (wd_set_batch_mode)
 * polls at most `polls` times before the solve gives up with WD_ERR_TIMEOUT.
 * 0 <= polls <= 2^26 (else WD_ERR_ARG); polls = 0 gives up at once, which
 * exercises the failure path without any fault.  Applies to the following
 * launches from this process.
 */
int wd_set_wait_limit(long long polls);

/*
 * Status of the asynchronous bounded waits on the current device: waits for
 * the work queued on the set stream, then returns WD_ERR_TIMEOUT if a launch
 * gave up waiting since the last call (and clears the flag), else WD_OK.
 * A raised flag means every launch since the previous call is untrustworthy.
 * Allocates nothing.
 */
int wd_async_status(void);

/* ------------------------------------------------------------------ */
/* solver (paper: even-odd preconditioned CG; Fig. 2)                  */
/* ------------------------------------------------------------------ */

typedef struct {
    int inner_prec;          /* WD_F64 (plain FP64 CG), WD_F32 or WD_F16 */
    int inner_recon;         /* link format of the inner operator: 12 or 18 */
    int outer_recon;         /* link format of the FP64 operator: 12 or 18 */
    int reliable_interval;   /* FP64 reliable update every n iterations (50) */
    int check_interval;      /* iterations between host convergence checks (10) */
    int maxiter;             /* iteration cap (default 100000) */
    int use_graph;           /* capture check_interval iterations as a CUDA graph */
    int use_initial_guess;   /* x holds a starting guess (restart / resume) */
    double tol;              /* target ||b - D x|| / ||b|| (default 1e-10) */
    int gauge_fix;           /* solve in temporal gauge (wd_gauge_fix_temporal) */
    int solver;              /* WD_SOLVER_CG (CG on the normal equations, default)
                                or WD_SOLVER_BICGSTAB (BiCGstab on the Schur
                                operator itself; the paper's second inverter) */
} wd_solve_params;

enum { WD_SOLVER_CG = 0, WD_SOLVER_BICGSTAB = 1 };

typedef struct {
    int iters;               /* inner iterations */
    int reliable_updates;    /* FP64 residual recomputations */
    int status;              /* WD_* */
    double true_residual;    /* ||b - D x|| / ||b||, FP64 on the full lattice */
    double seconds;          /* wall time of the solve inside wd_solve_ex */
    double dslash_calls;     /* hopping applications issued (all precisions) */
    double setup_seconds;    /* staging, packing, right-hand side, first residual */
    double iterate_seconds;  /* inner iterations (graph launches + checks) */
    double reliable_seconds; /* FP64 reliable updates inside the loop */
    double final_seconds;    /* odd-site reconstruction, true residual, unpack */
    int fallback_iters;      /* wd_solve_fcg: iterations of the plain-CG fallback
                                (0 when the preconditioned solve converged) */
} wd_solve_info;

/* Fill p with the defaults above (inner_prec WD_F32, recon 12 / 18). */
void wd_solve_params_default(wd_solve_params *p);

/*
 * Solve D x = b on the full lattice to ||b - D x||_2 / ||b||_2 <= tol, with
 * the even-odd Schur complement (1 - kappa^2 H_eo H_oe) x_e = b_e + kappa
 * H_eo b_o, CG on its normal equations (CGLS form), mixed precision with
 * FP64 reliable updates, then x_o = b_o + kappa H_oe x_e.
 * x, b: canonical FP64 full spinors; gauge: canonical FP64 gauge field.  Each
 * may be a host or a device pointer (detected per pointer); host data are
 * staged through library workspace.  Returns after the solve.
 */
int wd_solve(double *x, const double *b, const double *gauge, double kappa,
             double tol, const int dims[4]);

int wd_solve_ex(double *x, const double *b, const double *gauge, double kappa,
                const int dims[4], const wd_solve_params *params,
                wd_solve_info *info);

/*
 * Batched solves (many right-hand sides; several lattices, possibly of
 * different sizes).  Problem j solves D_j x = b for each of its nrhs
 * right-hand sides; b and x hold nrhs canonical FP64 full spinors back to
 * back (V_j * 24 doubles each), host or device memory; gauge is the
 * canonical FP64 gauge field of problem j.  Every right-hand side runs the
 * algorithm of wd_solve_ex with its own scalars and stops on its own
 * convergence; each iteration step is one launch over all problems and
 * right-hand sides (links reused across right-hand sides), and
 * check_interval iterations are one captured CUDA graph.
 * Limits: 1 <= nproblems <= 16, 1 <= nrhs <= 32 per problem; params->solver
 * must be WD_SOLVER_CG and params->gauge_fix 0 (else WD_ERR_ARG).
 * info (optional): one wd_solve_info per right-hand side, in problem order.
 * Returns WD_OK if every right-hand side converged, else the first failing
 * status (the per-right-hand-side statuses are in info).
 */
/*
 * Execution of the batched iterations (no counterpart in the paper).
 * mode = 0 (the default): one launch per step of the iteration (the four
 * hopping steps, the vector updates and the per-right-hand-side sums), with
 * the tile shapes of the autotuner.  mode = 1: every CG iteration of
 * wd_solve_batch is ONE persistent cooperative launch over all problems and
 * right-hand sides (one CTA per SM; the steps are phases separated by grid
 * barriers), for FP32 and FP16 inner iterations with 12-real links; other
 * inner formats run mode 0.  Every grid-barrier wait is bounded
 * (wd_set_wait_limit): a wait that runs out ends the solve with
 * WD_ERR_TIMEOUT and the context usable.  Both modes capture check_interval
 * iterations as a CUDA graph and give the same iterates up to the summation
 * order of the norms; on GB300 mode 0 is the faster (the hardware scheduler
 * balances the many small CTAs of each step; each phase of the persistent
 * launch waits at a grid barrier for its slowest warp).  Returns the previous
 * mode, or -WD_ERR_ARG for a mode other than 0 or 1.
 */
int wd_set_batch_mode(int mode);

typedef struct {
    int dims[4];
    double kappa;
    int nrhs;
    const double *gauge;
    const double *b;
    double *x;
} wd_batch_problem;

int wd_solve_batch(const wd_batch_problem *problems, int nproblems,
                   const wd_solve_params *params, wd_solve_info *info);

/* ------------------------------------------------------------------ */
/* learned preconditioner (not in the paper)                           */
/* ------------------------------------------------------------------ */

/*
 * A three-layer gauge-covariant nearest-neighbour network N, linear in its
 * input: layer l maps C_l -> C_{l+1} spin-like channels per colour
 * (4 -> 8 -> 8 -> 4, i.e. 12 -> 24 -> 24 -> 12 complex channels per site) as
 *     y(x)[o][a] = sum_{d=0..8} sum_i W_d[o][i] (T_d phi)(x)[i][a],
 * T_0 = identity, T_{1+2mu} phi(x) = U_mu(x) phi(x+mu),
 * T_{2+2mu} phi(x) = U_mu(x-mu)^+ phi(x-mu) (antiperiodic time sign as in D).
 * Weights: WD_NN_PARAMS floats, layers back to back, each [9][C_out][C_in]
 * complex (re, im), device memory.  The contraction runs on the tensor cores
 * (BF16 operands, FP32 accumulation); activations are FP32.
 */
enum { WD_NN_PARAMS = 2304 };

typedef struct {
    int samples;             /* training pairs (b = D x, x), x complex Gaussian (4096) */
    int batch;               /* pairs per Adam step (16) */
    int epochs;              /* passes over the samples (1) */
    float lr;                /* Adam learning rate (2e-3) */
    unsigned long long seed; /* seed of the on-device sample generator (4242) */
    int init;                /* 1: start from the hopping series (wd_nn_init) */
    int smooth;              /* k > 0: every other x is damped k times,
                              * x <- x - w D^+ D x with w = 1/(1+8 kappa)^2,
                              * which keeps the low modes of D that set the
                              * Krylov iteration count (0) */
} wd_nn_train_params;

typedef struct {
    int steps;
    double loss_first;       /* ||N(b) - x||^2 / ||x||^2 of the first step's last pair */
    double loss_last;        /* same for the last step */
    double seconds;
} wd_nn_train_info;

void wd_nn_train_params_default(wd_nn_train_params *p);

/* weights <- the truncated hopping series of D^-1:
 * N = (1 + kH)(1 + i kH)(1 - i kH) = 1 + kH + k^2 H^2 + k^3 H^3. */
int wd_nn_init(float *weights, double kappa);

/* One layer: out (cout channels) = sum_d W_d T_d in (cin channels),
 * cin, cout in {4, 8}; weights [9][cout][cin] complex (device).  Fields use
 * the packed FP32 full layout widened to C channels: per parity, blocks of
 * 32 sites holding 3C/2 16-byte groups per site (complex index c*3 + colour),
 * each half rounded up to 256 bytes; C = 4 is the packed FP32 spinor.
 * Synchronous. */
int wd_nn_layer(void *out, const void *in, const float *weights, int cin, int cout,
                const void *gauge, const int dims[4]);

/* Weight gradient of one layer (backpropagation):
 *     grad_d[o][i] = sum_{x, colour a} delta(x)[o][a] conj((T_d in)(x)[i][a])
 * in: cin channels, delta: cout channels (packed FP32 full layout as above);
 * grad: [9][cout][cin] complex FP32 (device).  The contraction runs on the
 * tensor cores (BF16 operands, FP32 accumulation); the per-CTA partial
 * gradients are summed in a fixed order.  (cin, cout) in {(4, 8), (8, 8),
 * (8, 4)}.  WD_ERR_TIMEOUT if a bounded device wait gave up.  Synchronous. */
int wd_nn_wgrad(float *grad, const void *in, const void *delta, int cin, int cout,
                const void *gauge, const int dims[4]);

/* Complex Gaussian spinor field written in the packed FP32 full layout:
 * component k of lexicographic site i is the complex normal number
 * first + 12 i + k of stream (seed, stream) of the counter-based SplitMix64 /
 * Box-Muller generator (Re, Im ~ N(0, 1/2)).  The training samples of
 * wd_nn_train are drawn this way. */
int wd_gaussian_spinor(void *out, unsigned long long seed, unsigned long long stream,
                       unsigned long long first, const int dims[4]);

/* out = N(in): packed FP32 full spinors (WD_FULL layout); gauge packed
 * WD_F32 with recon 12.  Synchronous. */
int wd_nn_apply(void *out, const void *in, const float *weights, const void *gauge,
                const int dims[4]);

/*
 * out = N(in) with options (flags, OR-ed; the paper has no such component):
 *   WD_NN_BF16  activations between the layers in BF16 (one bf16x2 per
 *               complex value), the link transport in packed bf16x2
 *               arithmetic, the channel mixing on the tensor cores with FP32
 *               accumulation: about twice as fast, with about 2^-8 relative
 *               rounding per layer.  in and out stay packed FP32 fields.
 *   WD_NN_EVEN  only the even-even block P_e N P_e: the odd half of in is
 *               taken as zero and never read, the odd half of out is not
 *               written (the first layer gives even sites only their self
 *               term and odd sites only their hops; the last layer computes
 *               the even sites only).
 * wd_solve_fcg applies N_e with both.  Synchronous; WD_ERR_ARG for other
 * flag bits.
 */
enum { WD_NN_BF16 = 1, WD_NN_EVEN = 2 };
int wd_nn_apply_ex(void *out, const void *in, const float *weights, const void *gauge,
                   const int dims[4], int flags);

/* Train N on pairs (D x, x) generated on the GPU (Adam, loss ||N(Dx) - x||^2).
 * gauge: canonical FP64 (host or device).  weights: device, in/out. */
int wd_nn_train(float *weights, const double *gauge, double kappa, const int dims[4],
                const wd_nn_train_params *params, wd_nn_train_info *info);

/*
 * Flexible GCR(m) on the full operator D x = b (restart length m <= 16),
 * right-preconditioned by N (weights may be NULL: plain GCR), FP32 inner
 * vectors with FP64 restarts: x accumulated and r = b - D x recomputed in FP64
 * at every restart; stops on ||b - D x|| / ||b|| <= params->tol.  x, b, gauge
 * canonical FP64, host or device.  info->reliable_updates counts restarts.
 */
int wd_solve_fgcr(double *x, const double *b, const double *gauge, double kappa,
                  const int dims[4], const float *weights, int m,
                  const wd_solve_params *params, wd_solve_info *info);

/*
 * Flexible CG on the even-odd preconditioned system (the paper's solver),
 * preconditioned by the network above (weights NULL: CG on the normal
 * equations of the even-odd system, no preconditioner).  The even-even block
 * of D^-1 is exactly the inverse of Mhat = 1 - kappa^2 H_eo H_oe, so the
 * even-even block N_e of a network trained as an approximate inverse of D
 * approximates Mhat^-1.  CG runs on Mhat^+ Mhat x_e = Mhat^+ bhat_e with the
 * preconditioner N_e N_e^+, which is Hermitian positive definite, so the
 * method converges where GCR on D stalls (kappa beyond the critical region of
 * the links, where the spectrum of D surrounds the origin); then
 * x_o = b_o + kappa H_oe x_e.  FP32 vectors and operator, BF16 network
 * arithmetic; the small variation of N's rounding between applications is
 * absorbed by the flexible (Polak-Ribiere) beta.  FP64 reliable updates
 * every params->reliable_interval iterations and whenever the FP32 residual
 * looks converged (x accumulated and r = bhat - Mhat x recomputed in FP64;
 * the search direction restarts).  Stops on ||b - D x|| / ||b|| <=
 * params->tol, computed in FP64 on the full lattice.  Plain CG is the
 * fallback: should the preconditioned iteration stop short (params->maxiter,
 * a non-finite residual, a network wait that timed out) the even-odd
 * mixed-precision CG of wd_solve_ex continues from its iterate
 * (info->fallback_iters > 0).  The preconditioner is an addition to the
 * paper.  x, b, gauge: canonical FP64, host or device.  info->reliable_updates
 * counts the FP64 residual recomputations.
 */
int wd_solve_fcg(double *x, const double *b, const double *gauge, double kappa,
                 const int dims[4], const float *weights, const wd_solve_params *params,
                 wd_solve_info *info);

#ifdef __cplusplus
}
#endif

#endif /* WD_H */
