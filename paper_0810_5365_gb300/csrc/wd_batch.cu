// Batched multi-right-hand-side solves: many right-hand sides on one gauge
// field, and several lattices of different sizes, advanced together.
//
// The algorithm per right-hand side is the one of wd_solver.cu (even-odd
// Schur complement, CGLS on its normal equations, FP32/FP16 inner
// iterations, FP64 reliable updates every `reliable_interval` iterations).
// What changes is the execution: every step of an iteration is ONE launch
// over all problems and right-hand sides (the multi-RHS hopping kernel of
// wd_mrhs.cuh reads each link from HBM once for all the right-hand sides of
// its problem; the BLAS steps walk the same tile list), CG scalars are per
// right-hand side on the device, a convergence mask switches finished
// right-hand sides off, and each block of `check_interval` iterations is one
// captured CUDA graph.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "wd_mrhs.cuh"

namespace wd {

cudaError_t launch_mrhs_f64(const MrhsBatch& bt, int recon, bool dagger, const int* active,
                            RedScratch rs, bool norm, int lanes, cudaStream_t st);
cudaError_t launch_mrhs_f32(const MrhsBatch& bt, int recon, bool dagger, const int* active,
                            RedScratch rs, bool norm, int lanes, cudaStream_t st);
cudaError_t launch_mrhs_f16(const MrhsBatch& bt, int recon, bool dagger, const int* active,
                            RedScratch rs, bool norm, int lanes, cudaStream_t st);

// Per-right-hand-side sums of the partials that a reducing batch kernel left
// in [local rhs][unit] layout (unit = tile or sub-tile, `stride` units per
// rhs row): problem j owns units s0[j] .. s0[j] + n[j] - 1.  One block per
// batch-wide right-hand side; each thread sums a fixed strided subset, then a
// fixed tree, so the result does not depend on scheduling.
struct SumList {
  int nprob, stride;
  int rhs0[MRHS_MAX_PROBLEMS], nrhs[MRHS_MAX_PROBLEMS];
  int s0[MRHS_MAX_PROBLEMS], n[MRHS_MAX_PROBLEMS];
};

constexpr int SUM_BS = 512;

__global__ void __launch_bounds__(SUM_BS) sum_partials_kernel(const __grid_constant__ SumList L,
                                                              const int* active,
                                                              const double* __restrict__ partials,
                                                              double* out) {
  __shared__ double red[SUM_BS / 32];
  const int gi = blockIdx.x;
  int j = -1;
  for (int k = 0; k < L.nprob; k++)
    if (gi >= L.rhs0[k] && gi < L.rhs0[k] + L.nrhs[k]) j = k;
  if (j < 0 || (active != nullptr && active[gi] == 0)) return;  // uniform per block
  const int r = gi - L.rhs0[j];
  const double* row = partials + (size_t)r * L.stride + L.s0[j];
  // four independent chains per thread keep four loads in flight; they are
  // combined in a fixed order
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int t = threadIdx.x;
  for (; t + 3 * SUM_BS < L.n[j]; t += 4 * SUM_BS) {
    a0 += __ldcg(row + t);
    a1 += __ldcg(row + t + SUM_BS);
    a2 += __ldcg(row + t + 2 * SUM_BS);
    a3 += __ldcg(row + t + 3 * SUM_BS);
  }
  for (; t < L.n[j]; t += SUM_BS) a0 += __ldcg(row + t);
  double v[1] = {(a0 + a1) + (a2 + a3)};
  block_sum<1, SUM_BS>(v, red);
  if (threadIdx.x == 0) out[gi] = v[0];
}

template <typename B>
static cudaError_t sum_partials(const B& bt, int units_per_tile, const int* active,
                                const double* partials, double* out, cudaStream_t st) {
  SumList L;
  std::memset(&L, 0, sizeof(L));
  L.nprob = bt.nprob;
  L.stride = bt.ntiles * units_per_tile;
  int nr = 0;
  for (int j = 0; j < bt.nprob; j++) {
    L.rhs0[j] = bt.p[j].rhs0;
    L.nrhs[j] = bt.p[j].nrhs;
    L.s0[j] = bt.p[j].tile0 * units_per_tile;
    L.n[j] = bt.p[j].ntiles * units_per_tile;
    nr = bt.p[j].rhs0 + bt.p[j].nrhs > nr ? bt.p[j].rhs0 + bt.p[j].nrhs : nr;
  }
  if (nr < 1) return cudaSuccess;
  sum_partials_kernel<<<nr, SUM_BS, 0, st>>>(L, active, partials, out);
  return cudaGetLastError();
}

static cudaError_t launch_mrhs_raw(int prec, const MrhsBatch& bt, int recon, bool dagger,
                                   const int* active, RedScratch rs, double* norm_out, int lanes,
                                   cudaStream_t st) {
  const bool norm = norm_out != nullptr;
  cudaError_t e = cudaErrorInvalidValue;
  switch (prec) {
    case WD_F64: e = launch_mrhs_f64(bt, recon, dagger, active, rs, norm, lanes, st); break;
    case WD_F32: e = launch_mrhs_f32(bt, recon, dagger, active, rs, norm, lanes, st); break;
    case WD_F16: e = launch_mrhs_f16(bt, recon, dagger, active, rs, norm, lanes, st); break;
  }
  if (e != cudaSuccess || !norm) return e;
  return sum_partials(bt, MRHS_BS / MRHS_SUB, active, rs.partials, norm_out, st);
}

// ---------------------------------------------------------------------------
// Autotuner of the multi-right-hand-side tile shape.  A batch shape (precision,
// link format, dagger, fused norm, tile count, largest nrhs, problem count)
// met for the first time outside stream capture is timed with every shape
// (1, 2, 4, 8 right-hand-side warps per CTA with one right-hand side per
// thread; for FP32 also 1, 2, 4 warps with two right-hand sides per thread,
// shape codes MRHS_PAIR + warps): one warm-up and three timed launches each,
// CUDA events on the launching stream, outputs (and norms) redirected to a
// temporary buffer so that no caller data is written.  The fastest shape is
// kept for the life of the process.
// ---------------------------------------------------------------------------

namespace {

struct MrhsKey {
  int prec, recon, dagger, norm, ntiles, maxr, nprob;
  bool operator<(const MrhsKey& o) const {
    const int a[7] = {prec, recon, dagger, norm, ntiles, maxr, nprob};
    const int b[7] = {o.prec, o.recon, o.dagger, o.norm, o.ntiles, o.maxr, o.nprob};
    for (int k = 0; k < 7; k++)
      if (a[k] != b[k]) return a[k] < b[k];
    return false;
  }
};

constexpr int NSHAPES = 7;
constexpr int SHAPE_CHOICES[NSHAPES] = {1, 2, 4, 8, MRHS_PAIR + 1, MRHS_PAIR + 2, MRHS_PAIR + 4};

struct MrhsTuned {
  int lanes;         // the chosen shape code
  float us[NSHAPES];  // per candidate, 0 when not timed
};

bool valid_shape(int shape) {
  for (int c = 0; c < NSHAPES; c++)
    if (SHAPE_CHOICES[c] == shape) return true;
  return false;
}

std::map<MrhsKey, MrhsTuned>& tune_table() {
  static std::map<MrhsKey, MrhsTuned> t;
  return t;
}
int g_autotune = 1;
int g_force_lanes = 0;

MrhsKey make_key(int prec, const MrhsBatch& bt, int recon, bool dagger, bool norm) {
  int maxr = 1;
  for (int j = 0; j < bt.nprob; j++) maxr = bt.p[j].nrhs > maxr ? bt.p[j].nrhs : maxr;
  return MrhsKey{prec, recon, dagger ? 1 : 0, norm ? 1 : 0, bt.ntiles, maxr, bt.nprob};
}

// The tuned (or default) shape for this batch; times the candidates when the
// shape is new, tuning is on and the stream is not being captured.
cudaError_t mrhs_lanes(int prec, const MrhsBatch& bt, int recon, bool dagger, const int* active,
                       RedScratch rs, bool norm, cudaStream_t st, int* lanes) {
  if (g_force_lanes) {
    // the pair shapes exist for FP32 only; other precisions take the
    // one-per-thread shape with the same warps
    *lanes = (g_force_lanes & MRHS_PAIR) && prec != WD_F32 ? g_force_lanes - MRHS_PAIR
                                                            : g_force_lanes;
    return cudaSuccess;
  }
  const MrhsKey key = make_key(prec, bt, recon, dagger, norm);
  auto it = tune_table().find(key);
  if (it != tune_table().end()) {
    *lanes = it->second.lanes;
    return cudaSuccess;
  }
  *lanes = MRHS_LANES;
  if (!g_autotune) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return cudaSuccess;
  // temporary outputs: every problem's nrhs fields, and the norms
  size_t total = 256 + (size_t)MRHS_MAX_PROBLEMS * MRHS_MAX * sizeof(double);
  for (int j = 0; j < bt.nprob; j++) total += ((size_t)bt.p[j].nrhs * bt.p[j].s_out + 255) / 256 * 256;
  char* buf = nullptr;
  if (cudaMalloc(&buf, total) != cudaSuccess) {
    cudaGetLastError();  // no room to tune: keep the default shape
    return cudaSuccess;
  }
  MrhsBatch t = bt;
  size_t off = 256 + (size_t)MRHS_MAX_PROBLEMS * MRHS_MAX * sizeof(double);
  for (int j = 0; j < bt.nprob; j++) {
    t.p[j].out = buf + off;
    // x and y keep pointing at the caller's fields: they are only read
    off += ((size_t)bt.p[j].nrhs * bt.p[j].s_out + 255) / 256 * 256;
  }
  double* nt = norm ? (double*)(buf + 256) : nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MrhsTuned best{MRHS_LANES, {}};
  float best_us = 0.f;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int c = 0; c < NSHAPES && e == cudaSuccess; c++) {
    const int L = SHAPE_CHOICES[c];
    if ((L & MRHS_PAIR) && prec != WD_F32) continue;
    e = launch_mrhs_raw(prec, t, recon, dagger, active, rs, nt, L, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int k = 0; k < 3 && e == cudaSuccess; k++)
      e = launch_mrhs_raw(prec, t, recon, dagger, active, rs, nt, L, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    const float us = ms * 1e3f / 3.f;
    best.us[c] = us;
    if (best_us == 0.f || us < best_us) {
      best_us = us;
      best.lanes = L;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t fe = cudaFree(buf);
  if (e != cudaSuccess) return e;
  if (fe != cudaSuccess) return fe;
  tune_table()[key] = best;
  *lanes = best.lanes;
  return cudaSuccess;
}

}  // namespace

static cudaError_t launch_mrhs(int prec, const MrhsBatch& bt, int recon, bool dagger,
                               const int* active, RedScratch rs, double* norm_out, cudaStream_t st) {
  int lanes = MRHS_LANES;
  cudaError_t e = mrhs_lanes(prec, bt, recon, dagger, active, rs, norm_out != nullptr, st, &lanes);
  if (e != cudaSuccess) return e;
  return launch_mrhs_raw(prec, bt, recon, dagger, active, rs, norm_out, lanes, st);
}

int set_autotune(int enable) {
  const int prev = g_autotune;
  g_autotune = enable ? 1 : 0;
  return prev;
}

int autotune_enabled() { return g_autotune; }

namespace {
int g_launch_overlap = 1;  // hopping kernels as programmatic dependent launches
}  // namespace

int launch_overlap() { return g_launch_overlap; }

int set_launch_overlap(int enable) {
  const int prev = g_launch_overlap;
  g_launch_overlap = enable ? 1 : 0;
  return prev;
}

namespace {
int g_dslash_block = 0;  // forced CTA size of the single-field hopping kernel (0: tuned)
std::vector<std::string>& dslash_lines() {
  static std::vector<std::string> v;
  return v;
}
}  // namespace

int dslash_forced_block() { return g_dslash_block; }

int dslash_set_block(int bs) {
  if (bs != 0 && bs != 64 && bs != 128 && bs != 256) return WD_ERR_ARG;
  g_dslash_block = bs;
  return WD_OK;
}

void dslash_tune_record(const char* line) { dslash_lines().push_back(line); }

int mrhs_set_lanes(int lanes) {
  if (lanes != 0 && !valid_shape(lanes)) return WD_ERR_ARG;
  g_force_lanes = lanes;
  return WD_OK;
}

int tune_report(char* buf, size_t len) {
  size_t used = 0;
  if (buf && len) buf[0] = 0;
  for (const auto& kv : tune_table()) {
    const MrhsKey& k = kv.first;
    const MrhsTuned& v = kv.second;
    char line[256];
    std::snprintf(line, sizeof(line),
                  "mrhs prec=%d recon=%d dagger=%d norm=%d tiles=%d maxrhs=%d problems=%d "
                  "us[1,2,4,8,p1,p2,p4]=%.1f,%.1f,%.1f,%.1f,%.1f,%.1f,%.1f shape=%s%d\n",
                  k.prec, k.recon, k.dagger, k.norm, k.ntiles, k.maxr, k.nprob, v.us[0], v.us[1],
                  v.us[2], v.us[3], v.us[4], v.us[5], v.us[6], (v.lanes & MRHS_PAIR) ? "p" : "",
                  v.lanes & ~MRHS_PAIR);
    const size_t n = std::strlen(line);
    if (buf && used + n + 1 <= len) {
      std::memcpy(buf + used, line, n + 1);
      used += n;
    }
  }
  for (const std::string& l : dslash_lines()) {
    if (buf && used + l.size() + 1 <= len) {
      std::memcpy(buf + used, l.c_str(), l.size() + 1);
      used += l.size();
    }
  }
  return (int)(tune_table().size() + dslash_lines().size());
}

// tune a launch shape without running it (before a graph capture)
static cudaError_t tune_mrhs(int prec, const MrhsBatch& bt, int recon, bool dagger,
                             const int* active, RedScratch rs, bool norm, cudaStream_t st) {
  int lanes = MRHS_LANES;
  return mrhs_lanes(prec, bt, recon, dagger, active, rs, norm, st, &lanes);
}

// ---------------------------------------------------------------------------
// batched BLAS over the same tile list
// ---------------------------------------------------------------------------

struct BlasProblem {
  Geom g;
  int nrhs, rhs0, tile0, ntiles;
  char* f[3];
  size_t s[3];
};

struct BlasBatch {
  int nprob, ntiles;
  BlasProblem p[MRHS_MAX_PROBLEMS];
};

#define WD_TILE_LOOP                                                   \
  for (int tile = blockIdx.x; tile < bt.ntiles; tile += gridDim.x) {   \
    int j = 0;                                                         \
    while (j + 1 < bt.nprob && tile >= bt.p[j + 1].tile0) j++;         \
    const BlasProblem& pr = bt.p[j];                                   \
    const int cb = (tile - pr.tile0) * MRHS_BS + threadIdx.x;          \
    const bool valid = cb < pr.g.Vh;                                   \
    const int VP = pr.g.Vh_pad;

// r -= alpha q (f0 = r, f1 = q); alpha = gk / qq per rhs; per-(rhs, tile)
// partials of ||r||^2, summed into rr by sum_partials_kernel
template <int P>
__global__ void __launch_bounds__(MRHS_BS) batch_update_r(const __grid_constant__ BlasBatch bt, const int* active,
                                                          const double* gk, const double* qq,
                                                          RedScratch rs, double* rr) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  (void)rr;
  __shared__ R red[MRHS_BS / 32];
  WD_TILE_LOOP
  for (int r = 0; r < pr.nrhs; r++) {
    const int gi = pr.rhs0 + r;
    if (active[gi] == 0) continue;
    R t = (R)0;
    if (valid) {
      const R alpha = (R)(gk[gi] / qq[gi]);
      char* fr = pr.f[0] + r * pr.s[0];
      const char* fq = pr.f[1] + r * pr.s[1];
      cx<R> a[12], b[12];
      load_spinor_rw<P, R>(a, fr, cb, VP);
      load_spinor_rw<P, R>(b, fq, cb, VP);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        a[k].r = fma(-alpha, b[k].r, a[k].r);
        a[k].i = fma(-alpha, b[k].i, a[k].i);
      }
      store_spinor<P, R>(fr, cb, VP, a);
      t = site_norm2<R>(a);
    }
    R v[1] = {t};
    block_sum<1, MRHS_BS, R>(v, red);
    if (threadIdx.x == 0) rs.partials[(size_t)r * bt.ntiles + tile] = (double)v[0];
  }
  }
}

// x += alpha p ; p = s + beta p   (f0 = x [PX], f1 = p, f2 = s)
template <int P, int PX>
__global__ void __launch_bounds__(MRHS_BS) batch_update_xp(const __grid_constant__ BlasBatch bt, const int* active,
                                                           const double* gk, const double* gk1,
                                                           const double* qq) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  using RX = typename std::conditional<PX == WD_F64, double, float>::type;
  WD_TILE_LOOP
  if (!valid) continue;
  for (int r = 0; r < pr.nrhs; r++) {
    const int gi = pr.rhs0 + r;
    if (active[gi] == 0) continue;
    const RX alpha = (RX)(gk[gi] / qq[gi]);
    const R beta = (R)(gk1[gi] / gk[gi]);
    char* fx = pr.f[0] + r * pr.s[0];
    char* fp = pr.f[1] + r * pr.s[1];
    const char* fs = pr.f[2] + r * pr.s[2];
    cx<R> pv[12], sv[12];
    cx<RX> xv[12];
    load_spinor_rw<P, R>(pv, fp, cb, VP);
    load_spinor_rw<P, R>(sv, fs, cb, VP);
    load_spinor_rw<PX, RX>(xv, fx, cb, VP);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      xv[k].r = fma(alpha, (RX)pv[k].r, xv[k].r);
      xv[k].i = fma(alpha, (RX)pv[k].i, xv[k].i);
      pv[k].r = fma(beta, pv[k].r, sv[k].r);
      pv[k].i = fma(beta, pv[k].i, sv[k].i);
    }
    store_spinor<PX, RX>(fx, cb, VP, xv);
    store_spinor<P, R>(fp, cb, VP, pv);
  }
  }
}

// x64 += xs ; xs = 0   (f0 = x64 even half, f1 = xs [PX])
template <int PX>
__global__ void __launch_bounds__(MRHS_BS) batch_ru_accumulate(const __grid_constant__ BlasBatch bt,
                                                               const int* active) {
  using RX = typename std::conditional<PX == WD_F64, double, float>::type;
  WD_TILE_LOOP
  if (!valid) continue;
  for (int r = 0; r < pr.nrhs; r++) {
    if (active[pr.rhs0 + r] == 0) continue;
    char* fx = pr.f[0] + r * pr.s[0];
    char* fs = pr.f[1] + r * pr.s[1];
    cx<double> a[12];
    cx<RX> b[12];
    load_spinor_rw<WD_F64, double>(a, fx, cb, VP);
    load_spinor_rw<PX, RX>(b, fs, cb, VP);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      a[k].r += (double)b[k].r;
      a[k].i += (double)b[k].i;
      b[k] = mk<RX>(0, 0);
    }
    store_spinor<WD_F64, double>(fx, cb, VP, a);
    store_spinor<PX, RX>(fs, cb, VP, b);
  }
  }
}

// dst = src (f0 = dst [PD], f1 = src [PS])
template <int PD, int PS>
__global__ void __launch_bounds__(MRHS_BS) batch_convert(const __grid_constant__ BlasBatch bt, const int* active) {
  using R = typename std::conditional<PD == WD_F64 || PS == WD_F64, double, float>::type;
  WD_TILE_LOOP
  if (!valid) continue;
  for (int r = 0; r < pr.nrhs; r++) {
    if (active[pr.rhs0 + r] == 0) continue;
    cx<R> v[12];
    load_spinor_rw<PS, R>(v, pr.f[1] + r * pr.s[1], cb, VP);
    store_spinor<PD, R>(pr.f[0] + r * pr.s[0], cb, VP, v);
  }
  }
}
#undef WD_TILE_LOOP

// ---------------------------------------------------------------------------
// One persistent launch per batched CG iteration.
//
// The steps of an iteration (the four multi-right-hand-side hopping steps,
// the two vector updates and the per-right-hand-side reductions) run as
// phases of one cooperative kernel whose CTAs are all resident, separated by
// grid barriers.  Work items are (32-site sub-tile, right-hand side), one
// warp each, in the order of the multi-RHS kernel (the right-hand sides of a
// sub-tile are adjacent, so a link comes from memory once for all of them).
// Reductions are deterministic: each warp sums its items' values per
// right-hand side in item order, each CTA sums its warps in order, and the
// CTA partials ([rhs][CTA]) are summed in CTA order by one warp per
// right-hand side.  Every barrier wait is bounded: a CTA whose wait runs out
// raises the error word and leaves; the others see it at their next wait and
// leave too, and the host reports WD_ERR_TIMEOUT.
// ---------------------------------------------------------------------------

// Warps per CTA, one CTA per SM, so that few CTAs meet at each grid barrier
// and each CTA can sum the per-CTA partials of a norm by itself: 24 for FP16
// (80 registers) and 20 for FP32, whose hopping code inside the kernel's
// item loop needs 96 registers to stay (nearly) free of spills.
template <int P>
struct PiWarps {
  static constexpr int value = P == WD_F32 ? 20 : 24;
};

struct IterPlan {
  MrhsBatch oe_p, eo_q, oe_r_dag, eo_s_dag;  // ts = H p ; q = p - k^2 H ts ; and the H^+ pair
  BlasBatch upd_r, upd_xp;                   // r -= alpha q ; x += alpha p, p = s + beta p
  int nr;                                    // right-hand sides in the batch
  int maxr;                                  // largest nrhs of a problem
};

struct GridBarrier {
  unsigned count;
  unsigned gen;
  int err;    // set by a CTA whose bounded wait ran out
  int pad;
};

// The plan of the running batched solve.  Constant memory, like the batch
// descriptors of the per-step kernels (kernel parameters): read-only to the
// kernel, so its fields are reloaded at will instead of held in registers.
// One plan per process: batched solves do not overlap (the library is used
// from one host thread, and wd_solve_batch returns after its solve).
__constant__ IterPlan c_pi_plan;

struct IterArgs {
  const int* active;
  const double* gk;   // gamma of this iteration (per rhs)
  double* gk1;        // gamma of the next iteration (written by CTA 0)
  double* qq;         // ||q||^2 (written by CTA 0)
  double* rr;         // ||r||^2 (written by CTA 0)
  double* partA;      // CTA partials [rhs][CTA]: ||q||^2, then ||s||^2
  double* partB;      // CTA partials of ||r||^2
  GridBarrier* bar;
  long spin_limit;
};

// all CTAs arrive before any leaves; false (and the CTA should return) if
// this CTA's bounded wait ran out or another CTA's did
__device__ __forceinline__ bool grid_barrier(GridBarrier* b, long limit) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 1;
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->err;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long spins = 0;
      while (*vgen == g0) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (spins++ >= limit) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (*verr) ok = 0;
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename B>
__device__ __forceinline__ int batch_problem(const B& bt, int tile) {
  int j = 0;
  while (j + 1 < bt.nprob && tile >= bt.p[j + 1].tile0) j++;
  return j;
}

// The work items of a phase are (32-site sub-tile, right-hand side slot
// r < maxr), the slots of a sub-tile consecutive; item i goes to global warp
// i mod (CTAs x warps), so a CTA's warps share the links of a sub-tile.
struct PiItem {
  int j;     // problem
  int r;     // right-hand side within the problem
  int cb;    // checkerboard site of this lane
  bool act;  // an active right-hand side of this problem at a real site
};

template <typename B>
__device__ __forceinline__ PiItem pi_item(const B& bt, int it, int maxr, const int* active) {
  constexpr int SUBS = MRHS_BS / MRHS_SUB;
  PiItem w;
  const int sub = it / maxr;
  w.r = it - sub * maxr;
  const int tile = sub / SUBS, q = sub - tile * SUBS;
  w.j = batch_problem(bt, tile);
  const auto& pr = bt.p[w.j];
  w.cb = (tile - pr.tile0) * MRHS_BS + q * MRHS_SUB + (int)threadIdx.x;
  w.act = w.r < pr.nrhs && active[pr.rhs0 + w.r] != 0;
  return w;
}

// the warps' per-right-hand-side accumulators (shared memory, [warp][rhs])
// -> the CTA's partials [rhs][CTA], warps summed in order; accumulators reset
template <int NW>
__device__ __forceinline__ void flush_partials(double* acc, int nr, double* part) {
  __syncthreads();
  const int t = threadIdx.y * 32 + threadIdx.x;
  for (int g = t; g < nr; g += NW * 32) {
    double v = 0.0;
    for (int w = 0; w < NW; w++) {
      v += acc[w * nr + g];
      acc[w * nr + g] = 0.0;
    }
    part[(size_t)g * gridDim.x + blockIdx.x] = v;
  }
}

// red[g] = sum over CTAs of part[g][CTA] in CTA order, computed by every CTA
// for itself (one warp per right-hand side), so all CTAs hold the same value
// without another grid barrier; CTA 0 also stores it in out[g].
template <int NW>
__device__ __forceinline__ void reduce_partials(const double* part, int nr, const int* active,
                                                double* red, double* out) {
  const int lane = threadIdx.x;
  for (int g = threadIdx.y; g < nr; g += NW) {
    if (active[g] == 0) continue;
    double v = 0.0;
    for (int c = lane; c < (int)gridDim.x; c += 32) v += __ldcg(part + (size_t)g * gridDim.x + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      red[g] = v;
      if (blockIdx.x == 0) out[g] = v;
    }
  }
  __syncthreads();
}

// one hopping phase over all items; NORM: ||out||^2 per rhs into acc
// COH: the input field was written earlier in this launch (coherent loads;
// the first step's input p is rewritten only after three grid barriers, so
// the read-only path serves it)
template <int P, int RC, bool DAG, bool NORM, int NW, bool COH>
__device__ __forceinline__ void pi_dslash_phase(const MrhsBatch& bt, int maxr, const int* active,
                                                double* acc, int nr) {
  constexpr int SUBS = MRHS_BS / MRHS_SUB;
  const int items = bt.ntiles * SUBS * maxr;
  const int stride = gridDim.x * NW;
  for (int it = blockIdx.x * NW + threadIdx.y; it < items; it += stride) {
    const PiItem w = pi_item(bt, it, maxr, active);
    const MrhsProblem& pr = bt.p[w.j];
    real_of<P> nrm = 0;
    if (w.act && w.cb < pr.g.Vh) nrm = mrhs_site<P, RC, DAG, NORM, COH>(pr, w.cb, w.r);
    if constexpr (NORM) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      if (threadIdx.x == 0 && w.act) acc[threadIdx.y * nr + pr.rhs0 + w.r] += nrm;
    }
  }
}

// r -= alpha q with ||r||^2 per rhs into acc (f0 = r, f1 = q); qq: the
// CTA's copy of the reduced ||q||^2
template <int P, int NW>
__device__ __forceinline__ void pi_update_r(const BlasBatch& bt, int maxr, const int* active,
                                            const double* gk, const double* qq, double* acc,
                                            int nr) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  constexpr int SUBS = MRHS_BS / MRHS_SUB;
  const int items = bt.ntiles * SUBS * maxr;
  const int stride = gridDim.x * NW;
  for (int it = blockIdx.x * NW + threadIdx.y; it < items; it += stride) {
    const PiItem w = pi_item(bt, it, maxr, active);
    const BlasProblem& pr = bt.p[w.j];
    const int gi = pr.rhs0 + w.r;
    R t = (R)0;
    if (w.act && w.cb < pr.g.Vh) {
      const int VP = pr.g.Vh_pad, cb = w.cb;
      const R alpha = (R)(gk[gi] / qq[gi]);
      char* fr = pr.f[0] + w.r * pr.s[0];
      const char* fq = pr.f[1] + w.r * pr.s[1];
      cx<R> a[12], b[12];
      load_spinor_rw<P, R>(a, fr, cb, VP);
      load_spinor_rw<P, R>(b, fq, cb, VP);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        a[k].r = fma(-alpha, b[k].r, a[k].r);
        a[k].i = fma(-alpha, b[k].i, a[k].i);
      }
      store_spinor<P, R>(fr, cb, VP, a);
      t = site_norm2<R>(a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0 && w.act) acc[threadIdx.y * nr + gi] += t;
  }
}

// x += alpha p ; p = s + beta p  (f0 = x [PX], f1 = p, f2 = s); qq, gk1:
// the CTA's copies of the reduced scalars
template <int P, int PX, int NW>
__device__ __forceinline__ void pi_update_xp(const BlasBatch& bt, int maxr, const int* active,
                                             const double* gk, const double* gk1,
                                             const double* qq) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  using RX = typename std::conditional<PX == WD_F64, double, float>::type;
  constexpr int SUBS = MRHS_BS / MRHS_SUB;
  const int items = bt.ntiles * SUBS * maxr;
  const int stride = gridDim.x * NW;
  for (int it = blockIdx.x * NW + threadIdx.y; it < items; it += stride) {
    const PiItem w = pi_item(bt, it, maxr, active);
    const BlasProblem& pr = bt.p[w.j];
    if (!(w.act && w.cb < pr.g.Vh)) continue;
    const int gi = pr.rhs0 + w.r, VP = pr.g.Vh_pad, cb = w.cb;
    const RX alpha = (RX)(gk[gi] / qq[gi]);
    const R beta = (R)(gk1[gi] / gk[gi]);
    char* fx = pr.f[0] + w.r * pr.s[0];
    char* fp = pr.f[1] + w.r * pr.s[1];
    const char* fs = pr.f[2] + w.r * pr.s[2];
    cx<R> pv[12], sv[12];
    cx<RX> xv[12];
    load_spinor_rw<P, R>(pv, fp, cb, VP);
    load_spinor_rw<P, R>(sv, fs, cb, VP);
    load_spinor_rw<PX, RX>(xv, fx, cb, VP);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      xv[k].r = fma(alpha, (RX)pv[k].r, xv[k].r);
      xv[k].i = fma(alpha, (RX)pv[k].i, xv[k].i);
      pv[k].r = fma(beta, pv[k].r, sv[k].r);
      pv[k].i = fma(beta, pv[k].i, sv[k].i);
    }
    store_spinor<PX, RX>(fx, cb, VP, xv);
    store_spinor<P, R>(fp, cb, VP, pv);
  }
}

// Dynamic shared memory of the persistent kernel: the warps' accumulators
// [NW][nr] and the CTA's reduced scalars qq, gamma_next, rr [3][nr].
__host__ __device__ constexpr size_t pi_smem_doubles(int nw, int nr) {
  return (size_t)(nw + 3) * nr;
}

// One CGLS iteration of every active right-hand side of the batch (the
// algorithm of batch_iteration_t, one launch, five grid barriers).
template <int P, int PX, int RC>
__global__ void __launch_bounds__(PiWarps<P>::value * 32, 1)
    batch_iteration_kernel(const IterArgs A) {
  constexpr int NW = PiWarps<P>::value;
  extern __shared__ double pi_smem[];
  const IterPlan& pl = c_pi_plan;
  const int nr = pl.nr, maxr = pl.maxr;
  double* acc = pi_smem;
  double* s_qq = pi_smem + (size_t)NW * nr;
  double* s_g1 = s_qq + nr;
  double* s_rr = s_g1 + nr;
  for (int t = threadIdx.y * 32 + threadIdx.x; t < NW * nr; t += NW * 32)
    acc[t] = 0.0;
  __syncthreads();
  // q = Mhat p with ||q||^2
  pi_dslash_phase<P, RC, false, false, NW, false>(pl.oe_p, maxr, A.active, acc, nr);
  if (!grid_barrier(A.bar, A.spin_limit)) return;
  pi_dslash_phase<P, RC, false, true, NW, true>(pl.eo_q, maxr, A.active, acc, nr);
  flush_partials<NW>(acc, nr, A.partA);
  if (!grid_barrier(A.bar, A.spin_limit)) return;
  // r -= alpha q with ||r||^2
  reduce_partials<NW>(A.partA, nr, A.active, s_qq, A.qq);
  pi_update_r<P, NW>(pl.upd_r, maxr, A.active, A.gk, s_qq, acc, nr);
  flush_partials<NW>(acc, nr, A.partB);
  if (!grid_barrier(A.bar, A.spin_limit)) return;
  // s = Mhat^+ r with ||s||^2
  pi_dslash_phase<P, RC, true, false, NW, true>(pl.oe_r_dag, maxr, A.active, acc, nr);
  if (!grid_barrier(A.bar, A.spin_limit)) return;
  pi_dslash_phase<P, RC, true, true, NW, true>(pl.eo_s_dag, maxr, A.active, acc, nr);
  flush_partials<NW>(acc, nr, A.partA);
  if (!grid_barrier(A.bar, A.spin_limit)) return;
  // x += alpha p ; p = s + beta p
  reduce_partials<NW>(A.partA, nr, A.active, s_g1, A.gk1);
  reduce_partials<NW>(A.partB, nr, A.active, s_rr, A.rr);
  pi_update_xp<P, PX, NW>(pl.upd_xp, maxr, A.active, A.gk, s_g1, s_qq);
}

// ---------------------------------------------------------------------------
// the batched solver
// ---------------------------------------------------------------------------

struct BatchProblemWs {
  int dims[4];
  double kappa;
  int nrhs, rhs0, tile0, ntiles;
  Geom g;
  void* g64 = nullptr;
  void* gs = nullptr;
  char* b64 = nullptr;   // nrhs full FP64 fields (even, odd)
  char* x64 = nullptr;   // nrhs full FP64
  char* rf64 = nullptr;  // nrhs full FP64
  char* bhat = nullptr;  // nrhs even FP64
  char* r64 = nullptr;   // nrhs even FP64
  char* t64 = nullptr;   // nrhs odd FP64
  char* p = nullptr;     // nrhs sloppy even
  char* q = nullptr;
  char* r = nullptr;
  char* s = nullptr;
  char* ts = nullptr;    // nrhs sloppy odd (H p)
  char* ts2 = nullptr;   // nrhs sloppy odd (H^+ r): a buffer of its own, so that no field
                         // is read at neighbours, rewritten and read again in one iteration
  char* xs = nullptr;    // nrhs sloppy-x even
  double* canon = nullptr;  // staging for host b / x (nrhs full canonical)
  double* canon_gauge = nullptr;
};

struct BatchScalars {
  double* gamma[2];
  double* qq;
  double* rr;
  double* r64;
  double* bnorm2;
  double* res_e;
  double* res_o;
};

namespace {

struct BatchCtx {
  std::vector<BatchProblemWs> pw;
  int nr = 0, sprec = WD_F32, srecon = 12, orecon = 18, xprec = WD_F32;
  double* scal = nullptr;     // 8 * nr doubles
  double* scal_h = nullptr;   // pinned copy
  int* active = nullptr;      // device mask
  int* active_h = nullptr;    // pinned
  BatchScalars sc;
  cudaStream_t cap = nullptr;
  std::vector<void*> allocs;
  double dslash_calls = 0;
};

void free_ctx(BatchCtx& c) {
  for (void* p : c.allocs) cudaFree(p);
  c.allocs.clear();
  if (c.scal_h) cudaFreeHost(c.scal_h);
  if (c.active_h) cudaFreeHost(c.active_h);
  if (c.cap) cudaStreamDestroy(c.cap);
  c.scal_h = nullptr;
  c.active_h = nullptr;
  c.cap = nullptr;
}

cudaError_t dalloc(BatchCtx& c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) c.allocs.push_back(*p);
  return e;
}

MrhsProblem mproblem(const BatchProblemWs& w, int parity, const void* gauge, double a, void* out,
                     size_t s_out, const void* in, size_t s_in, const void* x, size_t s_x,
                     double bx, const void* y, size_t s_y, double cy) {
  MrhsProblem m;
  std::memset(&m, 0, sizeof(m));
  m.g = w.g;
  m.gauge = gauge;
  m.nrhs = w.nrhs;
  m.rhs0 = w.rhs0;
  m.tile0 = w.tile0;
  m.ntiles = w.ntiles;
  m.parity = parity;
  m.a = a;
  m.bx = bx;
  m.cy = cy;
  m.out = out;
  m.in = in;
  m.x = x;
  m.y = y;
  m.s_out = s_out;
  m.s_in = s_in;
  m.s_x = s_x;
  m.s_y = s_y;
  return m;
}

BlasProblem bproblem(const BatchProblemWs& w, char* f0, size_t s0, char* f1, size_t s1,
                     char* f2 = nullptr, size_t s2 = 0) {
  BlasProblem b;
  std::memset(&b, 0, sizeof(b));
  b.g = w.g;
  b.nrhs = w.nrhs;
  b.rhs0 = w.rhs0;
  b.tile0 = w.tile0;
  b.ntiles = w.ntiles;
  b.f[0] = f0;
  b.f[1] = f1;
  b.f[2] = f2;
  b.s[0] = s0;
  b.s[1] = s1;
  b.s[2] = s2;
  return b;
}

// the batch descriptors of every step, built once per solve
struct Plan {
  MrhsBatch d_oe_p, d_eo_q, d_oe_r_dag, d_eo_s_dag;  // sloppy operator steps
  MrhsBatch r_t64, r_r64;                            // FP64 residual
  MrhsBatch bhat, xo, rf_e, rf_o;                    // FP64 setup / final
  BlasBatch upd_r, upd_xp, ru, cvt_r, cvt_p;
  int ntiles;
};

void build_plan(BatchCtx& c, Plan& pl) {
  std::memset(&pl, 0, sizeof(pl));
  const int np = (int)c.pw.size();
  MrhsBatch* ms[] = {&pl.d_oe_p, &pl.d_eo_q, &pl.d_oe_r_dag, &pl.d_eo_s_dag, &pl.r_t64,
                     &pl.r_r64,  &pl.bhat,   &pl.xo,         &pl.rf_e,       &pl.rf_o};
  BlasBatch* bs[] = {&pl.upd_r, &pl.upd_xp, &pl.ru, &pl.cvt_r, &pl.cvt_p};
  int nt = 0;
  for (auto& w : c.pw) nt = w.tile0 + w.ntiles;
  pl.ntiles = nt;
  for (MrhsBatch* m : ms) { m->nprob = np; m->ntiles = nt; }
  for (BlasBatch* b : bs) { b->nprob = np; b->ntiles = nt; }
  for (int j = 0; j < np; j++) {
    BatchProblemWs& w = c.pw[j];
    const double k = w.kappa, k2 = k * k;
    const size_t h64 = spinor_half_bytes(w.g, WD_F64);
    const size_t hs = spinor_half_bytes(w.g, c.sprec);
    const size_t hx = spinor_half_bytes(w.g, c.xprec);
    const size_t f64 = 2 * h64;  // full FP64 field
    // sloppy operator: ts = H_oe p ; q = p - k^2 H_eo ts ; and the dagger pair on r -> s
    pl.d_oe_p.p[j] = mproblem(w, WD_ODD, w.gs, 1.0, w.ts, hs, w.p, hs, nullptr, 0, 0, nullptr, 0, 0);
    pl.d_eo_q.p[j] = mproblem(w, WD_EVEN, w.gs, -k2, w.q, hs, w.ts, hs, w.p, hs, 1.0, nullptr, 0, 0);
    pl.d_oe_r_dag.p[j] = mproblem(w, WD_ODD, w.gs, 1.0, w.ts2, hs, w.r, hs, nullptr, 0, 0, nullptr, 0, 0);
    pl.d_eo_s_dag.p[j] = mproblem(w, WD_EVEN, w.gs, -k2, w.s, hs, w.ts2, hs, w.r, hs, 1.0, nullptr, 0, 0);
    // FP64: t64 = H_oe x_e ; r64 = k^2 H_eo t64 - x_e + bhat
    pl.r_t64.p[j] = mproblem(w, WD_ODD, w.g64, 1.0, w.t64, h64, w.x64, f64, nullptr, 0, 0, nullptr, 0, 0);
    pl.r_r64.p[j] = mproblem(w, WD_EVEN, w.g64, k2, w.r64, h64, w.t64, h64, w.x64, f64, -1.0, w.bhat, h64, 1.0);
    // bhat = b_e + k H_eo b_o
    pl.bhat.p[j] = mproblem(w, WD_EVEN, w.g64, k, w.bhat, h64, w.b64 + h64, f64, w.b64, f64, 1.0, nullptr, 0, 0);
    // x_o = b_o + k H_oe x_e ; rf_e = k H_eo x_o + b_e - x_e ; rf_o = k H_oe x_e + b_o - x_o
    pl.xo.p[j] = mproblem(w, WD_ODD, w.g64, k, w.x64 + h64, f64, w.x64, f64, w.b64 + h64, f64, 1.0, nullptr, 0, 0);
    pl.rf_e.p[j] = mproblem(w, WD_EVEN, w.g64, k, w.rf64, f64, w.x64 + h64, f64, w.b64, f64, 1.0, w.x64, f64, -1.0);
    pl.rf_o.p[j] = mproblem(w, WD_ODD, w.g64, k, w.rf64 + h64, f64, w.x64, f64, w.b64 + h64, f64, 1.0, w.x64 + h64, f64, -1.0);
    pl.upd_r.p[j] = bproblem(w, w.r, hs, w.q, hs);
    pl.upd_xp.p[j] = bproblem(w, w.xs, hx, w.p, hs, w.s, hs);
    pl.ru.p[j] = bproblem(w, w.x64, f64, w.xs, hx);
    pl.cvt_r.p[j] = bproblem(w, w.r, hs, w.r64, h64);
    pl.cvt_p.p[j] = bproblem(w, w.p, hs, w.s, hs);
  }
}

int blas_grid_tiles(int ntiles) {
  int g = num_sms() * 6;
  return ntiles < g ? (ntiles > 0 ? ntiles : 1) : g;
}

template <int P, int PX>
cudaError_t batch_iteration_t(BatchCtx& c, const Plan& pl, int kp, cudaStream_t st) {
  RedScratch rs = scratch();
  const BatchScalars& sc = c.sc;
  cudaError_t e;
  const int grid = blas_grid_tiles(pl.ntiles);
  c.dslash_calls += 4;
  if ((e = launch_mrhs(c.sprec, pl.d_oe_p, c.srecon, false, c.active, rs, nullptr, st))) return e;
  if ((e = launch_mrhs(c.sprec, pl.d_eo_q, c.srecon, false, c.active, rs, sc.qq, st))) return e;
  batch_update_r<P><<<grid, MRHS_BS, 0, st>>>(pl.upd_r, c.active, sc.gamma[kp], sc.qq, rs, sc.rr);
  if ((e = cudaGetLastError())) return e;
  if ((e = sum_partials(pl.upd_r, 1, c.active, rs.partials, sc.rr, st))) return e;
  if ((e = launch_mrhs(c.sprec, pl.d_oe_r_dag, c.srecon, true, c.active, rs, nullptr, st))) return e;
  if ((e = launch_mrhs(c.sprec, pl.d_eo_s_dag, c.srecon, true, c.active, rs, sc.gamma[1 - kp], st)))
    return e;
  batch_update_xp<P, PX><<<grid, MRHS_BS, 0, st>>>(pl.upd_xp, c.active, sc.gamma[kp],
                                                   sc.gamma[1 - kp], sc.qq);
  return cudaGetLastError();
}

cudaError_t batch_iteration(BatchCtx& c, const Plan& pl, int kp, cudaStream_t st) {
  switch (c.sprec) {
    case WD_F64: return batch_iteration_t<WD_F64, WD_F64>(c, pl, kp, st);
    case WD_F32: return batch_iteration_t<WD_F32, WD_F32>(c, pl, kp, st);
    case WD_F16: return batch_iteration_t<WD_F16, WD_F32>(c, pl, kp, st);
  }
  return cudaErrorInvalidValue;
}

// ---- the persistent iteration launch ----

// 0 (default): a launch per step; 1: one persistent launch per iteration.
// On GB300 the per-step launches are measured faster (12 right-hand sides
// on 24^3x48: 1.53 against 1.83 ms per FP32 iteration, 1.23 against 1.46 ms
// FP16): the hardware block scheduler balances the many small CTAs of each
// step, while the phases of the persistent kernel each end at a grid
// barrier that waits for its slowest warp.
int g_batch_mode = 0;

struct Persist {
  bool on = false;
  GridBarrier* bar = nullptr;
  double* partA = nullptr;
  double* partB = nullptr;
  int grid = 0;
  size_t smem = 0;
};

template <int P, int PX>
cudaError_t pi_launch(const Persist& ps, const BatchCtx& c, int kp, cudaStream_t st) {
  IterArgs A;
  A.active = c.active;
  A.gk = c.sc.gamma[kp];
  A.gk1 = c.sc.gamma[1 - kp];
  A.qq = c.sc.qq;
  A.rr = c.sc.rr;
  A.partA = ps.partA;
  A.partB = ps.partB;
  A.bar = ps.bar;
  A.spin_limit = state().wait_limit;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ps.grid);
  cfg.blockDim = dim3(32, PiWarps<P>::value);
  cfg.dynamicSmemBytes = ps.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_iteration_kernel<P, PX, 12>, A);
}

cudaError_t persist_launch(const Persist& ps, const BatchCtx& c, int kp, cudaStream_t st) {
  switch (c.sprec) {
    case WD_F32: return pi_launch<WD_F32, WD_F32>(ps, c, kp, st);
    case WD_F16: return pi_launch<WD_F16, WD_F32>(ps, c, kp, st);
  }
  return cudaErrorInvalidValue;
}

// the grid of the cooperative launch: every CTA the SMs hold at once
template <int P, int PX>
cudaError_t pi_grid(size_t smem, int* grid) {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, batch_iteration_kernel<P, PX, 12>, PiWarps<P>::value * 32, smem);
  if (e != cudaSuccess) return e;
  *grid = nb * num_sms();
  return cudaSuccess;
}

// set up the persistent path when the inner precision and link format have
// an instantiation; ps.on stays false otherwise (the per-step graph is used)
cudaError_t persist_setup(Persist& ps, BatchCtx& c, const Plan& pl, cudaStream_t st) {
  ps.on = false;
  if (g_batch_mode != 1 || c.srecon != 12 || (c.sprec != WD_F32 && c.sprec != WD_F16))
    return cudaSuccess;
  int dev = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) return e;
  ps.smem = pi_smem_doubles(c.sprec == WD_F32 ? PiWarps<WD_F32>::value : PiWarps<WD_F16>::value,
                            c.nr) * sizeof(double);
  {
    cudaError_t ea = c.sprec == WD_F32
        ? cudaFuncSetAttribute(batch_iteration_kernel<WD_F32, WD_F32, 12>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps.smem)
        : cudaFuncSetAttribute(batch_iteration_kernel<WD_F16, WD_F32, 12>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps.smem);
    if (ea != cudaSuccess) return ea;
  }
  e = c.sprec == WD_F32 ? pi_grid<WD_F32, WD_F32>(ps.smem, &ps.grid)
                        : pi_grid<WD_F16, WD_F32>(ps.smem, &ps.grid);
  if (e != cudaSuccess || ps.grid < 1) return e;
  IterPlan h;
  std::memset(&h, 0, sizeof(h));
  h.oe_p = pl.d_oe_p;
  h.eo_q = pl.d_eo_q;
  h.oe_r_dag = pl.d_oe_r_dag;
  h.eo_s_dag = pl.d_eo_s_dag;
  h.upd_r = pl.upd_r;
  h.upd_xp = pl.upd_xp;
  h.nr = c.nr;
  h.maxr = 1;
  for (auto& w : c.pw) h.maxr = w.nrhs > h.maxr ? w.nrhs : h.maxr;
  void* v;
  if ((e = dalloc(c, &v, sizeof(GridBarrier)))) return e;
  ps.bar = (GridBarrier*)v;
  if ((e = dalloc(c, &v, (size_t)c.nr * ps.grid * sizeof(double)))) return e;
  ps.partA = (double*)v;
  if ((e = dalloc(c, &v, (size_t)c.nr * ps.grid * sizeof(double)))) return e;
  ps.partB = (double*)v;
  if ((e = cudaMemcpyToSymbolAsync(c_pi_plan, &h, sizeof(h), 0, cudaMemcpyHostToDevice, st)))
    return e;
  if ((e = cudaMemsetAsync(ps.bar, 0, sizeof(GridBarrier), st))) return e;
  // a plan on the host stack: wait for the copy before it goes out of scope
  if ((e = cudaStreamSynchronize(st))) return e;
  ps.on = true;
  return cudaSuccess;
}

template <int PD, int PS>
void convert_b(const BlasBatch& b, const int* active, int grid, cudaStream_t st) {
  batch_convert<PD, PS><<<grid, MRHS_BS, 0, st>>>(b, active);
}

cudaError_t batch_reliable_update(BatchCtx& c, const Plan& pl, bool accumulate, cudaStream_t st,
                                  bool x_is_zero = false) {
  RedScratch rs = scratch();
  const int grid = blas_grid_tiles(pl.ntiles);
  cudaError_t e;
  if (accumulate) {
    if (c.xprec == WD_F64)
      batch_ru_accumulate<WD_F64><<<grid, MRHS_BS, 0, st>>>(pl.ru, c.active);
    else
      batch_ru_accumulate<WD_F32><<<grid, MRHS_BS, 0, st>>>(pl.ru, c.active);
    if ((e = cudaGetLastError())) return e;
  }
  if (x_is_zero) {
    // a start from x = 0: r64 = bhat exactly, no FP64 operator needed
    c.dslash_calls += 2;
    for (int j = 0; j < pl.r_r64.nprob; j++) {
      const MrhsProblem& m = pl.r_r64.p[j];
      const char* bh = (const char*)m.y;  // bhat of this problem (rhs stride s_y)
      if ((e = cudaMemcpyAsync(m.out, bh, (size_t)m.nrhs * m.s_out, cudaMemcpyDeviceToDevice,
                               st)))
        return e;
      for (int r = 0; r < m.nrhs; r++)
        if ((e = norm2(c.sc.r64 + m.rhs0 + r, (const char*)m.out + (size_t)r * m.s_out, m.g,
                       WD_F64, 1, st)))
          return e;
    }
  } else {
    c.dslash_calls += 4;
    if ((e = launch_mrhs(WD_F64, pl.r_t64, c.orecon, false, c.active, rs, nullptr, st))) return e;
    if ((e = launch_mrhs(WD_F64, pl.r_r64, c.orecon, false, c.active, rs, c.sc.r64, st)))
      return e;
  }
  switch (c.sprec) {
    case WD_F64: convert_b<WD_F64, WD_F64>(pl.cvt_r, c.active, grid, st); break;
    case WD_F32: convert_b<WD_F32, WD_F64>(pl.cvt_r, c.active, grid, st); break;
    case WD_F16: convert_b<WD_F16, WD_F64>(pl.cvt_r, c.active, grid, st); break;
  }
  if ((e = cudaGetLastError())) return e;
  if ((e = launch_mrhs(c.sprec, pl.d_oe_r_dag, c.srecon, true, c.active, rs, nullptr, st))) return e;
  if ((e = launch_mrhs(c.sprec, pl.d_eo_s_dag, c.srecon, true, c.active, rs, c.sc.gamma[0], st)))
    return e;
  switch (c.sprec) {
    case WD_F64: convert_b<WD_F64, WD_F64>(pl.cvt_p, c.active, grid, st); break;
    case WD_F32: convert_b<WD_F32, WD_F32>(pl.cvt_p, c.active, grid, st); break;
    case WD_F16: convert_b<WD_F16, WD_F16>(pl.cvt_p, c.active, grid, st); break;
  }
  return cudaGetLastError();
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

#define WD_BCK(call)                          \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) {                  \
      state().last_cuda_error = (int)e_;      \
      free_ctx(c);                            \
      return WD_ERR_CUDA;                     \
    }                                         \
  } while (0)

int solve_batch_impl(const wd_batch_problem* probs, int nprob, const wd_solve_params* prm,
                     wd_solve_info* infos) {
  const auto t0 = std::chrono::steady_clock::now();
  auto secs = [&](std::chrono::steady_clock::time_point a) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
  };
  wd_solve_params P;
  wd_solve_params_default(&P);
  if (prm) P = *prm;
  if (P.inner_prec < WD_F64 || P.inner_prec > WD_F16) return WD_ERR_PREC;
  if (link_bytes(P.inner_prec, P.inner_recon) == 0 || link_bytes(WD_F64, P.outer_recon) == 0)
    return WD_ERR_PREC;
  if (!(P.tol > 0) || P.maxiter < 0 || P.reliable_interval < 1) return WD_ERR_ARG;
  if (P.solver != WD_SOLVER_CG || P.gauge_fix) return WD_ERR_ARG;  // batched CG only
  const int chunk = P.check_interval < 2 ? 2 : (P.check_interval & ~1);
  cudaStream_t st = state().stream;

  BatchCtx c;
  c.sprec = P.inner_prec;
  c.srecon = P.inner_recon;
  c.orecon = P.outer_recon;
  c.xprec = P.inner_prec == WD_F64 ? WD_F64 : WD_F32;
  int tile0 = 0, nr = 0;
  for (int j = 0; j < nprob; j++) {
    BatchProblemWs w;
    std::memcpy(w.dims, probs[j].dims, sizeof(w.dims));
    w.kappa = probs[j].kappa;
    w.nrhs = probs[j].nrhs;
    w.rhs0 = nr;
    w.g = make_geom(w.dims);
    w.tile0 = tile0;
    w.ntiles = (w.g.Vh + MRHS_BS - 1) / MRHS_BS;
    tile0 += w.ntiles;
    nr += w.nrhs;
    c.pw.push_back(w);
  }
  c.nr = nr;

  // ---- allocation ----
  for (auto& w : c.pw) {
    const size_t h64 = spinor_half_bytes(w.g, WD_F64), hs = spinor_half_bytes(w.g, c.sprec);
    const size_t hx = spinor_half_bytes(w.g, c.xprec), n = (size_t)w.nrhs;
    WD_BCK(dalloc(c, &w.g64, gauge_bytes(w.g, WD_F64, c.orecon)));
    if (c.sprec == WD_F64 && c.srecon == c.orecon)
      w.gs = w.g64;
    else
      WD_BCK(dalloc(c, &w.gs, gauge_bytes(w.g, c.sprec, c.srecon)));
    void* v;
    WD_BCK(dalloc(c, &v, n * 2 * h64)); w.b64 = (char*)v;
    WD_BCK(dalloc(c, &v, n * 2 * h64)); w.x64 = (char*)v;
    WD_BCK(dalloc(c, &v, n * 2 * h64)); w.rf64 = (char*)v;
    WD_BCK(dalloc(c, &v, n * h64)); w.bhat = (char*)v;
    WD_BCK(dalloc(c, &v, n * h64)); w.r64 = (char*)v;
    WD_BCK(dalloc(c, &v, n * h64)); w.t64 = (char*)v;
    WD_BCK(dalloc(c, &v, n * hs)); w.p = (char*)v;
    WD_BCK(dalloc(c, &v, n * hs)); w.q = (char*)v;
    WD_BCK(dalloc(c, &v, n * hs)); w.r = (char*)v;
    WD_BCK(dalloc(c, &v, n * hs)); w.s = (char*)v;
    WD_BCK(dalloc(c, &v, n * hs)); w.ts = (char*)v;
    WD_BCK(dalloc(c, &v, n * hs)); w.ts2 = (char*)v;
    WD_BCK(dalloc(c, &v, n * hx)); w.xs = (char*)v;
  }
  {
    void* v;
    WD_BCK(dalloc(c, &v, 8 * (size_t)nr * sizeof(double)));
    c.scal = (double*)v;
    WD_BCK(cudaMemsetAsync(c.scal, 0, 8 * (size_t)nr * sizeof(double), st));
    WD_BCK(cudaMallocHost(&c.scal_h, 8 * (size_t)nr * sizeof(double)));
    WD_BCK(dalloc(c, &v, (size_t)nr * sizeof(int)));
    c.active = (int*)v;
    WD_BCK(cudaMallocHost(&c.active_h, (size_t)nr * sizeof(int)));
    double* s = c.scal;
    c.sc.gamma[0] = s; c.sc.gamma[1] = s + nr; c.sc.qq = s + 2 * nr; c.sc.rr = s + 3 * nr;
    c.sc.r64 = s + 4 * nr; c.sc.bnorm2 = s + 5 * nr; c.sc.res_e = s + 6 * nr;
    c.sc.res_o = s + 7 * nr;
    WD_BCK(cudaStreamCreateWithFlags(&c.cap, cudaStreamNonBlocking));
    WD_BCK(ensure_scratch((size_t)tile0 * (MRHS_BS / MRHS_SUB) * MRHS_MAX + 4096));
  }
  for (int g = 0; g < nr; g++) c.active_h[g] = 1;
  WD_BCK(cudaMemcpyAsync(c.active, c.active_h, nr * sizeof(int), cudaMemcpyHostToDevice, st));

  // ---- stage and pack ----
  for (int j = 0; j < nprob; j++) {
    BatchProblemWs& w = c.pw[j];
    const size_t V = 2 * (size_t)w.g.Vh, fb = V * 24 * sizeof(double);
    const size_t h64 = spinor_half_bytes(w.g, WD_F64);
    const double* gd = probs[j].gauge;
    if (!dev_ptr(gd)) {
      void* v;
      WD_BCK(dalloc(c, &v, 4 * V * 18 * sizeof(double)));
      WD_BCK(cudaMemcpyAsync(v, gd, 4 * V * 18 * sizeof(double), cudaMemcpyHostToDevice, st));
      gd = (const double*)v;
    }
    WD_BCK(pack_gauge(w.g64, gd, w.g, WD_F64, c.orecon, st));
    if (w.gs != w.g64) WD_BCK(pack_gauge(w.gs, gd, w.g, c.sprec, c.srecon, st));
    const double* bd = probs[j].b;
    if (!dev_ptr(bd)) {
      void* v;
      WD_BCK(dalloc(c, &v, (size_t)w.nrhs * fb));
      w.canon = (double*)v;
      WD_BCK(cudaMemcpyAsync(w.canon, bd, (size_t)w.nrhs * fb, cudaMemcpyHostToDevice, st));
      bd = w.canon;
    }
    for (int r = 0; r < w.nrhs; r++) {
      WD_BCK(pack_spinor(w.b64 + r * 2 * h64, bd + (size_t)r * V * 24, w.g, WD_FULL, WD_F64, st));
      WD_BCK(norm2(c.sc.bnorm2 + w.rhs0 + r, w.b64 + r * 2 * h64, w.g, WD_F64, 2, st));
    }
    if (P.use_initial_guess) {
      const double* xd = probs[j].x;
      if (!dev_ptr(xd)) {
        if (!w.canon) {
          void* v;
          WD_BCK(dalloc(c, &v, (size_t)w.nrhs * fb));
          w.canon = (double*)v;
        }
        WD_BCK(cudaMemcpyAsync(w.canon, xd, (size_t)w.nrhs * fb, cudaMemcpyHostToDevice, st));
        xd = w.canon;
      }
      for (int r = 0; r < w.nrhs; r++)
        WD_BCK(pack_spinor(w.x64 + r * 2 * h64, xd + (size_t)r * V * 24, w.g, WD_FULL, WD_F64, st));
    } else {
      WD_BCK(cudaMemsetAsync(w.x64, 0, (size_t)w.nrhs * 2 * h64, st));
    }
    WD_BCK(cudaMemsetAsync(w.xs, 0, (size_t)w.nrhs * spinor_half_bytes(w.g, c.xprec), st));
  }
  Plan pl;
  build_plan(c, pl);
  {
    RedScratch rs = scratch();
    c.dslash_calls += 1;
    WD_BCK(launch_mrhs(WD_F64, pl.bhat, c.orecon, false, c.active, rs, nullptr, st));
  }
  WD_BCK(batch_reliable_update(c, pl, false, st, !P.use_initial_guess));
  auto read_scal = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(c.scal_h, c.scal, 8 * (size_t)nr * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
  };
  WD_BCK(read_scal());
  const double* H = c.scal_h;
  std::vector<double> target(nr);
  std::vector<int> status(nr, WD_ERR_NOCONV), iters(nr, 0), rus(nr, 0);
  int nact = 0;
  for (int g = 0; g < nr; g++) {
    double bn = std::sqrt(H[5 * nr + g]);
    target[g] = P.tol * bn * 0.9;
    if (!std::isfinite(bn)) {
      status[g] = WD_ERR_NONFINITE;
      c.active_h[g] = 0;
    } else if (!(bn > 0) || std::sqrt(H[4 * nr + g]) <= target[g]) {
      status[g] = WD_OK;
      c.active_h[g] = 0;
    } else {
      nact++;
    }
  }
  WD_BCK(cudaMemcpyAsync(c.active, c.active_h, nr * sizeof(int), cudaMemcpyHostToDevice, st));
  const double t_setup = secs(t0);

  // ---- the iteration graph ----
  Persist ps;
  WD_BCK(persist_setup(ps, c, pl, st));
  auto iteration = [&](int kp, cudaStream_t s) -> cudaError_t {
    return ps.on ? persist_launch(ps, c, kp, s) : batch_iteration(c, pl, kp, s);
  };
  cudaGraphExec_t exec = nullptr;
  if (P.use_graph && nact > 0) {
    // the inner launch shapes, tuned before they are frozen into the graph
    if (!ps.on) {
      RedScratch rs = scratch();
      WD_BCK(tune_mrhs(c.sprec, pl.d_oe_p, c.srecon, false, c.active, rs, false, st));
      WD_BCK(tune_mrhs(c.sprec, pl.d_eo_q, c.srecon, false, c.active, rs, true, st));
      WD_BCK(tune_mrhs(c.sprec, pl.d_oe_r_dag, c.srecon, true, c.active, rs, false, st));
      WD_BCK(tune_mrhs(c.sprec, pl.d_eo_s_dag, c.srecon, true, c.active, rs, true, st));
    }
    cudaGraph_t graph = nullptr;
    WD_BCK(cudaStreamBeginCapture(c.cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    const double calls = c.dslash_calls;
    for (int k = 0; k < chunk && ce == cudaSuccess; k++) ce = iteration(k & 1, c.cap);
    c.dslash_calls = calls;
    cudaError_t ee = cudaStreamEndCapture(c.cap, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      state().last_cuda_error = (int)(ce != cudaSuccess ? ce : ee);
      free_ctx(c);
      return WD_ERR_CUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      state().last_cuda_error = (int)ie;
      free_ctx(c);
      return WD_ERR_CUDA;
    }
  }

  int it = 0, last_ru = 0;
  double t_ru = 0.0;
  const auto t_loop = std::chrono::steady_clock::now();
  int err = WD_OK;
  while (nact > 0 && it < P.maxiter) {
    cudaError_t e;
    if (exec) {
      e = cudaGraphLaunch(exec, st);
      c.dslash_calls += 4.0 * chunk;
    } else {
      e = cudaSuccess;
      for (int k = 0; k < chunk && e == cudaSuccess; k++) e = iteration(k & 1, st);
    }
    if (e == cudaSuccess) e = read_scal();
    if (e != cudaSuccess) { state().last_cuda_error = (int)e; err = WD_ERR_CUDA; break; }
    if (ps.on) {
      // a grid barrier whose bounded wait ran out ends the solve
      GridBarrier hb;
      e = cudaMemcpy(&hb, ps.bar, sizeof(hb), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) { state().last_cuda_error = (int)e; err = WD_ERR_CUDA; break; }
      if (hb.err) { err = WD_ERR_TIMEOUT; break; }
    }
    it += chunk;
    bool any_done = false;
    for (int g = 0; g < nr; g++) {
      if (!c.active_h[g]) continue;
      iters[g] += chunk;
      const double rr = H[3 * nr + g], qq = H[2 * nr + g], ga = H[g];
      if (!std::isfinite(rr) || !std::isfinite(ga)) {
        status[g] = WD_ERR_NONFINITE;
        c.active_h[g] = 0;
        nact--;
      } else if (!(qq > 0) || !(ga > 0)) {
        status[g] = WD_ERR_BREAKDOWN;
        c.active_h[g] = 0;
        nact--;
      } else if (std::sqrt(rr) <= target[g]) {
        any_done = true;
      }
    }
    if (nact > 0 && (any_done || it - last_ru >= (c.sprec == WD_F64 ? 0x7fffffff : P.reliable_interval) ||
                     it >= P.maxiter)) {
      const auto ta = std::chrono::steady_clock::now();
      e = batch_reliable_update(c, pl, true, st);
      if (e == cudaSuccess) e = read_scal();
      t_ru += secs(ta);
      if (e != cudaSuccess) { state().last_cuda_error = (int)e; err = WD_ERR_CUDA; break; }
      last_ru = it;
      for (int g = 0; g < nr; g++) {
        if (!c.active_h[g]) continue;
        rus[g]++;
        const double r = std::sqrt(H[4 * nr + g]);
        if (!std::isfinite(r)) {
          status[g] = WD_ERR_NONFINITE;
          c.active_h[g] = 0;
          nact--;
        } else if (r <= target[g]) {
          status[g] = WD_OK;
          c.active_h[g] = 0;
          nact--;
        }
      }
    }
    e = cudaMemcpyAsync(c.active, c.active_h, nr * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { state().last_cuda_error = (int)e; err = WD_ERR_CUDA; break; }
  }
  if (exec) cudaGraphExecDestroy(exec);
  const double t_iter = secs(t_loop) - t_ru;
  if (err != WD_OK) {
    free_ctx(c);
    return err;
  }
  // right-hand sides still active at maxiter keep their last reliable update
  const auto t_fin = std::chrono::steady_clock::now();
  for (int g = 0; g < nr; g++) c.active_h[g] = 1;
  WD_BCK(cudaMemcpyAsync(c.active, c.active_h, nr * sizeof(int), cudaMemcpyHostToDevice, st));
  {
    RedScratch rs = scratch();
    c.dslash_calls += 3;
    WD_BCK(launch_mrhs(WD_F64, pl.xo, c.orecon, false, c.active, rs, nullptr, st));
    WD_BCK(launch_mrhs(WD_F64, pl.rf_e, c.orecon, false, c.active, rs, c.sc.res_e, st));
    WD_BCK(launch_mrhs(WD_F64, pl.rf_o, c.orecon, false, c.active, rs, c.sc.res_o, st));
  }
  for (int j = 0; j < nprob; j++) {
    BatchProblemWs& w = c.pw[j];
    const size_t V = 2 * (size_t)w.g.Vh, fb = V * 24 * sizeof(double);
    const size_t h64 = spinor_half_bytes(w.g, WD_F64);
    double* xo = probs[j].x;
    const bool xdev = dev_ptr(xo);
    double* dst = xdev ? xo : w.canon;
    if (!dst) {
      void* v;
      WD_BCK(dalloc(c, &v, (size_t)w.nrhs * fb));
      w.canon = (double*)v;
      dst = w.canon;
    }
    for (int r = 0; r < w.nrhs; r++)
      WD_BCK(unpack_spinor(dst + (size_t)r * V * 24, w.x64 + r * 2 * h64, w.g, WD_FULL, WD_F64, st));
    if (!xdev)
      WD_BCK(cudaMemcpyAsync(xo, dst, (size_t)w.nrhs * fb, cudaMemcpyDeviceToHost, st));
  }
  WD_BCK(read_scal());
  const double t_final = secs(t_fin);
  const double total = secs(t0);
  int worst = WD_OK;
  for (int g = 0; g < nr; g++) {
    const double bn = std::sqrt(H[5 * nr + g]);
    const double rel = bn > 0 ? std::sqrt(H[6 * nr + g] + H[7 * nr + g]) / bn : 0.0;
    if (status[g] == WD_OK && !(rel <= P.tol)) status[g] = WD_ERR_NOCONV;
    if (status[g] != WD_OK && worst == WD_OK) worst = status[g];
    if (infos) {
      wd_solve_info& I = infos[g];
      std::memset(&I, 0, sizeof(I));
      I.iters = iters[g];
      I.reliable_updates = rus[g];
      I.status = status[g];
      I.true_residual = rel;
      I.seconds = total;
      I.dslash_calls = c.dslash_calls;
      I.setup_seconds = t_setup;
      I.iterate_seconds = t_iter;
      I.reliable_seconds = t_ru;
      I.final_seconds = t_final;
    }
  }
  free_ctx(c);
  return worst;
}

int set_batch_mode(int mode) {
  const int prev = g_batch_mode;
  g_batch_mode = mode;
  return prev;
}

// single problem, many right-hand sides: one hopping application
cudaError_t dslash_mrhs(void* out, const void* in, const void* gauge, int parity, int dagger,
                        double a, const void* x, double bx, int nrhs, double* norms,
                        const Geom& g, int prec, int recon, cudaStream_t st) {
  MrhsBatch bt;
  std::memset(&bt, 0, sizeof(bt));
  bt.nprob = 1;
  bt.ntiles = (g.Vh + MRHS_BS - 1) / MRHS_BS;
  MrhsProblem& m = bt.p[0];
  const size_t h = spinor_half_bytes(g, prec);
  m.g = g;
  m.gauge = gauge;
  m.nrhs = nrhs;
  m.rhs0 = 0;
  m.tile0 = 0;
  m.ntiles = bt.ntiles;
  m.parity = parity;
  m.a = a;
  m.bx = bx;
  m.out = out;
  m.in = in;
  m.x = x;
  m.s_out = m.s_in = m.s_x = h;
  if (norms) {
    cudaError_t e = ensure_scratch((size_t)bt.ntiles * (MRHS_BS / MRHS_SUB) * MRHS_MAX + 1024);
    if (e != cudaSuccess) return e;
  }
  return launch_mrhs(prec, bt, recon, dagger != 0, nullptr, scratch(), norms, st);
}

}  // namespace wd
