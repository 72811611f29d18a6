// Multi-right-hand-side hopping kernel over a batch of problems.
//
// A batch is a list of problems (lattice geometry, gauge field, nrhs fields);
// the problems may have different lattice sizes.  Their sites of one parity
// are cut into tiles of MRHS_BS checkerboard sites and all tiles of all
// problems form one launch.  The warps of a CTA (1, 2, 4 or 8, chosen by the
// autotuner) apply the hopping term to different right-hand sides of the same
// 32 sites, and the CTAs covering the other right-hand sides of those sites
// are adjacent in launch order, so each link crosses HBM once per site instead
// of once per site and right-hand side (the repeats are served by L1/L2).
// Per right-hand side the epilogue is the one of the
// single-field kernel (out = a H in + bx x + cy y), optionally with ||out||^2
// reduced deterministically per right-hand side (per-sub-tile partials here,
// their fixed-order sum in sum_partials_kernel).
#pragma once

#include "wd_dslash.cuh"

namespace wd {

constexpr int MRHS_BS = 128;   // sites per tile = threads per CTA
constexpr int MRHS_MAX = 32;   // right-hand sides per problem

struct MrhsProblem {
  Geom g;
  const void* gauge;
  int nrhs;
  int rhs0;       // batch-wide index of the first right-hand side
  int tile0;      // first tile of this problem in the batch's tile range
  int ntiles;
  int parity;     // output parity
  double a, bx, cy;  // out = a H in + bx x + cy y
  void* out;
  const void* in;
  const void* x;  // may be null; may alias out
  const void* y;  // may be null; may alias out
  size_t s_out, s_in, s_x, s_y;  // bytes between consecutive right-hand sides
};

// The whole batch travels as one kernel parameter (under 4 KB), so a launch
// needs no descriptor upload and a captured graph keeps its own copy.
constexpr int MRHS_MAX_PROBLEMS = 16;
struct MrhsBatch {
  int nprob;
  int ntiles;
  MrhsProblem p[MRHS_MAX_PROBLEMS];
};

// One CTA = 32 sites x L right-hand-side lanes (one warp per right-hand
// side).  Block b covers sub-tile b / G and right-hand sides L (b % G) ..
// L (b % G) + L - 1, G = ceil(max nrhs / L): the G blocks of a sub-tile are
// adjacent in launch order, run together, and read the same links, which
// L1/L2 then return once per site for all right-hand sides.  Each thread
// computes one right-hand side of one site, so the kernel keeps the registers
// (and occupancy) of the single-field kernel.
constexpr int MRHS_LANES = 4;   // default right-hand-side lanes (warps) per CTA
constexpr int MRHS_SUB = 32;    // sites per CTA

// The tile shape is a template parameter (1, 2, 4 or 8 right-hand-side warps
// per CTA) chosen per batch shape by the autotuner; the register budget per
// thread is the single-field kernel's for every shape.
#ifndef WD_MRHS_MINB_F32_NORM
#define WD_MRHS_MINB_F32_NORM 7  // measured: 6% faster than 6 despite a small spill
#endif
template <int P, bool NORM>
struct MrhsMinBlocks4 {  // CTAs per SM the budget is sized for, at 4 lanes
  static constexpr int value =
      (P == WD_F32 && NORM) ? WD_MRHS_MINB_F32_NORM : DslashMinBlocks<P, NORM>::value;
};
template <int P, bool NORM, int LANES>
struct MrhsMinBlocks {
  static constexpr int raw = MrhsMinBlocks4<P, NORM>::value * MRHS_LANES / LANES;
  static constexpr int value = raw < 1 ? 1 : (raw > 32 ? 32 : raw);
};

// One right-hand side r of one site cb of problem pr: out = a H in + bx x +
// cy y, returning ||out||^2 at this site when NORM (else 0).  COH: the input
// field is read with coherent loads (it was written earlier in the launch).
template <int P, int RC, bool DAG, bool NORM, bool COH = false>
__device__ __forceinline__ real_of<P> mrhs_site(const MrhsProblem& pr, int cb, int r) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  constexpr int SF = DAG ? -1 : 1;
  constexpr int SB_ = -SF;
  const Geom& g = pr.g;
  const int p = pr.parity, qq = 1 - p, VP = g.Vh_pad;
  int x0, x1, x2, x3;
  cb_coords(cb, p, g, x0, x1, x2, x3);
  const int row = cb - (x0 >> 1);
  const int f0 = row + ((x0 + 1 == g.L[0] ? 0 : x0 + 1) >> 1);
  const int b0 = row + ((x0 == 0 ? g.L[0] - 1 : x0 - 1) >> 1);
  const int f1 = x1 == g.L[1] - 1 ? cb - (g.L[1] - 1) * g.S1 : cb + g.S1;
  const int b1 = x1 == 0 ? cb + (g.L[1] - 1) * g.S1 : cb - g.S1;
  const int f2 = x2 == g.L[2] - 1 ? cb - (g.L[2] - 1) * g.S2 : cb + g.S2;
  const int b2 = x2 == 0 ? cb + (g.L[2] - 1) * g.S2 : cb - g.S2;
  const int f3 = x3 == g.L[3] - 1 ? cb - (g.L[3] - 1) * g.S3 : cb + g.S3;
  const int b3 = x3 == 0 ? cb + (g.L[3] - 1) * g.S3 : cb - g.S3;
  const bool fflip = x3 == g.L[3] - 1;
  const bool bflip = x3 == 0;
  const void* in = (const char*)pr.in + (size_t)r * pr.s_in;
  const void* ga = pr.gauge;
  cx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
  void* out = (char*)pr.out + (size_t)r * pr.s_out;
  bool stored = false;
  if constexpr (P == WD_F16) {
    __half2 ah[12];
    const float kf = (float)pr.a * hops_f16<SF, SB_, COH>(ah, in, ga, p, cb, f0, b0, f1, b1, f2,
                                                         b2, f3, b3, fflip, bflip, false, false,
                                                         VP);
    if (!pr.x && !pr.y) {
      store_f16_h2<NORM>(out, cb, VP, ah, kf, acc);
      stored = true;
    } else {
      f16_widen(acc, ah, kf);
    }
  } else {
    hop<P, RC, 0, SF, true, R, COH>(acc, in, ga, f0, 0 + p, cb, false, VP);
    hop<P, RC, 0, SB_, false, R, COH>(acc, in, ga, b0, 0 + qq, b0, false, VP);
    hop<P, RC, 1, SF, true, R, COH>(acc, in, ga, f1, 2 + p, cb, false, VP);
    hop<P, RC, 1, SB_, false, R, COH>(acc, in, ga, b1, 2 + qq, b1, false, VP);
    hop<P, RC, 2, SF, true, R, COH>(acc, in, ga, f2, 4 + p, cb, false, VP);
    hop<P, RC, 2, SB_, false, R, COH>(acc, in, ga, b2, 4 + qq, b2, false, VP);
    hop<P, RC, 3, SF, true, R, COH>(acc, in, ga, f3, 6 + p, cb, fflip, VP);
    hop<P, RC, 3, SB_, false, R, COH>(acc, in, ga, b3, 6 + qq, b3, bflip, VP);
  }
  if constexpr (P != WD_F16) {  // (the FP16 hops apply a themselves)
    const R ca = (R)pr.a;
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = ca * acc[k];
  }
  if (!stored) {
    if (pr.x) {
      cx<R> v[12];
      load_spinor_rw<P, R>(v, (const char*)pr.x + (size_t)r * pr.s_x, cb, VP);
      const R cbx = (R)pr.bx;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[k].r = fma(cbx, v[k].r, acc[k].r);
        acc[k].i = fma(cbx, v[k].i, acc[k].i);
      }
    }
    if (pr.y) {
      cx<R> v[12];
      load_spinor_rw<P, R>(v, (const char*)pr.y + (size_t)r * pr.s_y, cb, VP);
      const R ccy = (R)pr.cy;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[k].r = fma(ccy, v[k].r, acc[k].r);
        acc[k].i = fma(ccy, v[k].i, acc[k].i);
      }
    }
    if constexpr (P == WD_F16 && NORM)
      store_spinor_f16<R, true>(out, cb, VP, acc);
    else
      store_spinor<P, R>(out, cb, VP, acc);
  }
  R nrm = (R)0;
  if constexpr (NORM) nrm = site_norm2<R>(acc);  // (FP16: acc holds what was stored)
  return nrm;
}

template <int P, int RC, bool DAG, bool NORM, int LANES>
__global__ void __launch_bounds__(MRHS_SUB* LANES, (MrhsMinBlocks<P, NORM, LANES>::value))
    mrhs_dslash_kernel(const __grid_constant__ MrhsBatch bt, int groups,
                       const int* __restrict__ active, RedScratch rs) {
  const int tx = threadIdx.x, ry = threadIdx.y;
  constexpr int SUBS = MRHS_BS / MRHS_SUB;  // sub-tiles per tile
  const int nprob = bt.nprob;
  const int sub = blockIdx.x / groups;
  const int r = (blockIdx.x - sub * groups) * LANES + ry;
  const int tile = sub / SUBS, q = sub - tile * SUBS;
  int j = 0;
  while (j + 1 < nprob && tile >= bt.p[j + 1].tile0) j++;
  const MrhsProblem& pr = bt.p[j];
  const int cb = (tile - pr.tile0) * MRHS_BS + q * MRHS_SUB + tx;
  const bool act = r < pr.nrhs && (active == nullptr || active[pr.rhs0 + r] != 0);
  real_of<P> nrm = 0;
  if (act && cb < pr.g.Vh) nrm = mrhs_site<P, RC, DAG, NORM>(pr, cb, r);
  if constexpr (NORM) {
    // one warp = one right-hand side of these 32 sites, summed in the
    // working precision; the per-(rhs, sub-tile) partials are FP64, summed
    // in a fixed order by sum_partials_kernel ([local rhs][sub-tile] layout,
    // so that those reads coalesce)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (tx == 0 && act) rs.partials[(size_t)r * (bt.ntiles * SUBS) + sub] = (double)nrm;
  }
}

// ---------------------------------------------------------------------------
// FP32 with two right-hand sides per thread.  The link of each hop is loaded
// and its third row rebuilt once, then multiplies the half spinors of both
// right-hand sides, so the L1 requests per right-hand-side site drop from
// 8 * 48 + 8 * 96 + 96 to 8 * 24 + 8 * 96 + 96 bytes and the link
// instructions are halved.  The price is registers: two accumulators.  Thread
// (x, y) of block b computes right-hand sides 2 (L (b % G) + y) and the next
// one, G = ceil(max nrhs / 2L).  When the second right-hand side does not
// exist or is masked off, the thread still computes it on the first one's
// field (branch-free, so both hops' loads can be in flight together) and
// discards it.
// ---------------------------------------------------------------------------
constexpr int MRHS_PAIR = 16;  // shape code bit: two right-hand sides per thread

#ifndef WD_MRHS2_MINB4
#define WD_MRHS2_MINB4 4  // CTAs per SM at 4 warps the pair kernel is budgeted for
#endif
template <int LANES>
struct Mrhs2MinBlocks {
  static constexpr int raw = WD_MRHS2_MINB4 * 4 / LANES;
  static constexpr int value = raw < 1 ? 1 : (raw > 32 ? 32 : raw);
};

template <int RC, int MU, int S, bool FWD>
__device__ __forceinline__ void hop_pair_f32(cx<float> (&a0)[12], cx<float> (&a1)[12],
                                             const void* __restrict__ in0,
                                             const void* __restrict__ in1,
                                             const void* __restrict__ gauge, int nb, int region,
                                             int lcb, bool flip, int VP) {
  cx<float> u[9];
  load_link<WD_F32, RC, float>(u, gauge, region, lcb, VP);
  cx<float> h0[6], h1[6];
  load_project<WD_F32, MU, S, float>(h0, in0, nb, VP);
  load_project<WD_F32, MU, S, float>(h1, in1, nb, VP);
  cx<float> t[6];
#if WD_F32X2
  su3_mul_f32x2<FWD>(u, h0, t);
#else
#error "the pair kernel uses the packed FP32 link product"
#endif
  if constexpr (MU == 3) {
    expand_add<MU, S, false>(a0, t, flip ? -1.f : 1.f);
  } else {
    expand_add<MU, S, true>(a0, t, 1.f);
  }
  su3_mul_f32x2<FWD>(u, h1, t);
  if constexpr (MU == 3) {
    expand_add<MU, S, false>(a1, t, flip ? -1.f : 1.f);
  } else {
    expand_add<MU, S, true>(a1, t, 1.f);
  }
}

// out = a H in + bx x + cy y for one right-hand side of one site (F32)
__device__ __forceinline__ void mrhs_epilogue_f32(cx<float> (&acc)[12], const MrhsProblem& pr,
                                                  int r, int cb, int VP) {
  const float ca = (float)pr.a;
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = ca * acc[k];
  if (pr.x) {
    cx<float> v[12];
    load_spinor_rw<WD_F32, float>(v, (const char*)pr.x + (size_t)r * pr.s_x, cb, VP);
    const float cbx = (float)pr.bx;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      acc[k].r = fmaf(cbx, v[k].r, acc[k].r);
      acc[k].i = fmaf(cbx, v[k].i, acc[k].i);
    }
  }
  if (pr.y) {
    cx<float> v[12];
    load_spinor_rw<WD_F32, float>(v, (const char*)pr.y + (size_t)r * pr.s_y, cb, VP);
    const float ccy = (float)pr.cy;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      acc[k].r = fmaf(ccy, v[k].r, acc[k].r);
      acc[k].i = fmaf(ccy, v[k].i, acc[k].i);
    }
  }
  store_spinor<WD_F32, float>((char*)pr.out + (size_t)r * pr.s_out, cb, VP, acc);
}

template <int RC, bool DAG, bool NORM, int LANES>
__global__ void __launch_bounds__(MRHS_SUB* LANES, (Mrhs2MinBlocks<LANES>::value))
    mrhs_pair_kernel(const __grid_constant__ MrhsBatch bt, int groups,
                     const int* __restrict__ active, RedScratch rs) {
  const int tx = threadIdx.x, ry = threadIdx.y;
  constexpr int SF = DAG ? -1 : 1;
  constexpr int SB_ = -SF;
  constexpr int SUBS = MRHS_BS / MRHS_SUB;
  const int nprob = bt.nprob;
  const int sub = blockIdx.x / groups;
  const int r0 = 2 * ((blockIdx.x - sub * groups) * LANES + ry), r1 = r0 + 1;
  const int tile = sub / SUBS, q = sub - tile * SUBS;
  int j = 0;
  while (j + 1 < nprob && tile >= bt.p[j + 1].tile0) j++;
  const MrhsProblem& pr = bt.p[j];
  const int cb = (tile - pr.tile0) * MRHS_BS + q * MRHS_SUB + tx;
  const bool act0 = r0 < pr.nrhs && (active == nullptr || active[pr.rhs0 + r0] != 0);
  const bool act1 = r1 < pr.nrhs && (active == nullptr || active[pr.rhs0 + r1] != 0);
  float nrm0 = 0.f, nrm1 = 0.f;
  if ((act0 || act1) && cb < pr.g.Vh) {
    const Geom& g = pr.g;
    const int p = pr.parity, qq = 1 - p, VP = g.Vh_pad;
    int x0, x1, x2, x3;
    cb_coords(cb, p, g, x0, x1, x2, x3);
    const int row = cb - (x0 >> 1);
    const int f0 = row + ((x0 + 1 == g.L[0] ? 0 : x0 + 1) >> 1);
    const int b0 = row + ((x0 == 0 ? g.L[0] - 1 : x0 - 1) >> 1);
    const int f1 = x1 == g.L[1] - 1 ? cb - (g.L[1] - 1) * g.S1 : cb + g.S1;
    const int b1 = x1 == 0 ? cb + (g.L[1] - 1) * g.S1 : cb - g.S1;
    const int f2 = x2 == g.L[2] - 1 ? cb - (g.L[2] - 1) * g.S2 : cb + g.S2;
    const int b2 = x2 == 0 ? cb + (g.L[2] - 1) * g.S2 : cb - g.S2;
    const int f3 = x3 == g.L[3] - 1 ? cb - (g.L[3] - 1) * g.S3 : cb + g.S3;
    const int b3 = x3 == 0 ? cb + (g.L[3] - 1) * g.S3 : cb - g.S3;
    const bool fflip = x3 == g.L[3] - 1;
    const bool bflip = x3 == 0;
    // an absent or masked right-hand side is computed on the other one's
    // field and discarded
    const int ra = act0 ? r0 : r1, rb = act1 ? r1 : r0;
    const void* in0 = (const char*)pr.in + (size_t)ra * pr.s_in;
    const void* in1 = (const char*)pr.in + (size_t)rb * pr.s_in;
    const void* ga = pr.gauge;
    cx<float> a0[12], a1[12];
#pragma unroll
    for (int k = 0; k < 12; k++) a0[k] = a1[k] = mk<float>(0.f, 0.f);
    hop_pair_f32<RC, 0, SF, true>(a0, a1, in0, in1, ga, f0, 0 + p, cb, false, VP);
    hop_pair_f32<RC, 0, SB_, false>(a0, a1, in0, in1, ga, b0, 0 + qq, b0, false, VP);
    hop_pair_f32<RC, 1, SF, true>(a0, a1, in0, in1, ga, f1, 2 + p, cb, false, VP);
    hop_pair_f32<RC, 1, SB_, false>(a0, a1, in0, in1, ga, b1, 2 + qq, b1, false, VP);
    hop_pair_f32<RC, 2, SF, true>(a0, a1, in0, in1, ga, f2, 4 + p, cb, false, VP);
    hop_pair_f32<RC, 2, SB_, false>(a0, a1, in0, in1, ga, b2, 4 + qq, b2, false, VP);
    hop_pair_f32<RC, 3, SF, true>(a0, a1, in0, in1, ga, f3, 6 + p, cb, fflip, VP);
    hop_pair_f32<RC, 3, SB_, false>(a0, a1, in0, in1, ga, b3, 6 + qq, b3, bflip, VP);
    if (act0) {
      mrhs_epilogue_f32(a0, pr, r0, cb, VP);
      if constexpr (NORM) nrm0 = site_norm2<float>(a0);
    }
    if (act1) {
      mrhs_epilogue_f32(a1, pr, r1, cb, VP);
      if constexpr (NORM) nrm1 = site_norm2<float>(a1);
    }
  }
  if constexpr (NORM) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nrm0 += __shfl_xor_sync(0xffffffffu, nrm0, o);
      nrm1 += __shfl_xor_sync(0xffffffffu, nrm1, o);
    }
    if (tx == 0 && act0) rs.partials[(size_t)r0 * (bt.ntiles * SUBS) + sub] = (double)nrm0;
    if (tx == 0 && act1) rs.partials[(size_t)r1 * (bt.ntiles * SUBS) + sub] = (double)nrm1;
  }
}

template <int RC, bool DG, bool NM, int L>
cudaError_t launch_mrhs_pair_one(const MrhsBatch& bt, const int* active, RedScratch rs,
                                 cudaStream_t st) {
  int maxr = 1;
  for (int j = 0; j < bt.nprob; j++) maxr = bt.p[j].nrhs > maxr ? bt.p[j].nrhs : maxr;
  const int groups = (maxr + 2 * L - 1) / (2 * L);
  const long long nblk = (long long)bt.ntiles * (MRHS_BS / MRHS_SUB) * groups;
  mrhs_pair_kernel<RC, DG, NM, L><<<(unsigned)nblk, dim3(MRHS_SUB, L), 0, st>>>(bt, groups,
                                                                              active, rs);
  return cudaGetLastError();
}

template <int RC, bool DG, bool NM>
cudaError_t launch_mrhs_pair(const MrhsBatch& bt, const int* active, RedScratch rs, int lanes,
                             cudaStream_t st) {
  switch (lanes) {
    case 1: return launch_mrhs_pair_one<RC, DG, NM, 1>(bt, active, rs, st);
    case 2: return launch_mrhs_pair_one<RC, DG, NM, 2>(bt, active, rs, st);
    case 4: return launch_mrhs_pair_one<RC, DG, NM, 4>(bt, active, rs, st);
  }
  return cudaErrorInvalidValue;
}

template <int P, int RC, bool DG, bool NM, int L>
cudaError_t launch_mrhs_one(const MrhsBatch& bt, const int* active, RedScratch rs,
                            cudaStream_t st) {
  int maxr = 1;
  for (int j = 0; j < bt.nprob; j++) maxr = bt.p[j].nrhs > maxr ? bt.p[j].nrhs : maxr;
  const int groups = (maxr + L - 1) / L;
  const long long nblk = (long long)bt.ntiles * (MRHS_BS / MRHS_SUB) * groups;
  mrhs_dslash_kernel<P, RC, DG, NM, L><<<(unsigned)nblk, dim3(MRHS_SUB, L), 0, st>>>(
      bt, groups, active, rs);
  return cudaGetLastError();
}

template <int P, int RC, bool DG, bool NM>
cudaError_t launch_mrhs_lanes(const MrhsBatch& bt, const int* active, RedScratch rs, int lanes,
                              cudaStream_t st) {
  if (lanes & MRHS_PAIR) {
    if constexpr (P == WD_F32) return launch_mrhs_pair<RC, DG, NM>(bt, active, rs,
                                                                    lanes - MRHS_PAIR, st);
    return cudaErrorInvalidValue;
  }
  switch (lanes) {
    case 1: return launch_mrhs_one<P, RC, DG, NM, 1>(bt, active, rs, st);
    case 2: return launch_mrhs_one<P, RC, DG, NM, 2>(bt, active, rs, st);
    case 4: return launch_mrhs_one<P, RC, DG, NM, 4>(bt, active, rs, st);
    case 8: return launch_mrhs_one<P, RC, DG, NM, 8>(bt, active, rs, st);
  }
  return cudaErrorInvalidValue;
}

// norm: the kernel leaves per-(rhs, sub-tile) partials of ||out||^2 in rs
template <int P>
cudaError_t launch_mrhs_prec(const MrhsBatch& bt, int recon, bool dagger, const int* active,
                             RedScratch rs, bool norm, int lanes, cudaStream_t st) {
  if (recon == 12) {
    if (dagger) return norm ? launch_mrhs_lanes<P, 12, true, true>(bt, active, rs, lanes, st)
                            : launch_mrhs_lanes<P, 12, true, false>(bt, active, rs, lanes, st);
    return norm ? launch_mrhs_lanes<P, 12, false, true>(bt, active, rs, lanes, st)
                : launch_mrhs_lanes<P, 12, false, false>(bt, active, rs, lanes, st);
  }
  if constexpr (P != WD_F16) {
    if (recon == 18) {
      if (dagger) return norm ? launch_mrhs_lanes<P, 18, true, true>(bt, active, rs, lanes, st)
                              : launch_mrhs_lanes<P, 18, true, false>(bt, active, rs, lanes, st);
      return norm ? launch_mrhs_lanes<P, 18, false, true>(bt, active, rs, lanes, st)
                  : launch_mrhs_lanes<P, 18, false, false>(bt, active, rs, lanes, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace wd
