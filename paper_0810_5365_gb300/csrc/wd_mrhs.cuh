// Multi-right-hand-side hopping kernel over a batch of problems.
//
// A batch is a list of problems (lattice geometry, gauge field, nrhs fields);
// the problems may have different lattice sizes.  Their sites of one parity
// are cut into tiles of MRHS_BS checkerboard sites and all tiles of all
// problems form one launch.  A CTA takes a tile, stages the eight links of
// each of its sites in shared memory once (12-real FP32 / FP16 formats), and
// then applies the hopping term to every active right-hand side of the
// problem, so each link crosses HBM once per site instead of once per site
// and right-hand side.  Per right-hand side the epilogue is the one of the
// single-field kernel (out = a H in + bx x + cy y), optionally with ||out||^2
// reduced deterministically per right-hand side.
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

// link slots staged per thread and hop (128-bit vectors)
template <int P, int RC>
struct MrhsStage {
  static constexpr bool on = (P == WD_F32 || P == WD_F16) && RC == 12;
  static constexpr int vec16 = P == WD_F32 ? 3 : 2;  // F16: int4 + int2 (padded to 16 B)
  static constexpr size_t bytes_per_thread = on ? 8 * vec16 * 16 : 0;
};

template <int P, int RC>
__device__ __forceinline__ void stage_link(int4* sm, int hop, int tid, const void* gauge,
                                           int region, int lcb, int VP) {
  if constexpr (P == WD_F32) {
    const int4* p = (const int4*)gauge + (size_t)region * VP * 3;
#pragma unroll
    for (int k = 0; k < 3; k++) sm[(hop * 3 + k) * MRHS_BS + tid] = __ldg(p + sbi(lcb, k, 3));
  } else {
    const int4* pa = (const int4*)gauge + (size_t)region * VP;
    const int2* pb = (const int2*)((const char*)gauge + (size_t)8 * VP * 16) + (size_t)region * VP;
    int2 b = __ldg(pb + lcb);
    sm[(hop * 2 + 0) * MRHS_BS + tid] = __ldg(pa + lcb);
    sm[(hop * 2 + 1) * MRHS_BS + tid] = make_int4(b.x, b.y, 0, 0);
  }
}

template <int P, typename R>
__device__ __forceinline__ void unstage_link(cx<R> (&u)[9], const int4* sm, int hop, int tid) {
  if constexpr (P == WD_F32) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      int4 w = sm[(hop * 3 + k) * MRHS_BS + tid];
      float4 v = *reinterpret_cast<const float4*>(&w);
      u[2 * k] = mk<R>(v.x, v.y);
      u[2 * k + 1] = mk<R>(v.z, v.w);
    }
  } else {
    int4 a = sm[(hop * 2 + 0) * MRHS_BS + tid];
    int4 b = sm[(hop * 2 + 1) * MRHS_BS + tid];
    const __half2* ha = reinterpret_cast<const __half2*>(&a);
    const __half2* hb = reinterpret_cast<const __half2*>(&b);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float2 f = __half22float2(ha[j]);
      u[j] = mk<R>(f.x, f.y);
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
      float2 f = __half22float2(hb[j]);
      u[4 + j] = mk<R>(f.x, f.y);
    }
  }
  reconstruct_row2(u);
}

// one hop with a link already in registers
template <int P, int MU, int S, bool FWD, typename R>
__device__ __forceinline__ void hop_with_link(cx<R> (&acc)[12], const void* __restrict__ in, int nb,
                                              const cx<R> (&u)[9], bool flip, int VP) {
  cx<R> h[6];
  R sc = load_project<P, MU, S, R>(h, in, nb, VP);
  cx<R> t[6];
#pragma unroll
  for (int hs = 0; hs < 2; hs++) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      cx<R> v = mk<R>(0, 0);
#pragma unroll
      for (int d = 0; d < 3; d++) {
        if (FWD)
          v = cmadd(u[c * 3 + d], h[hs * 3 + d], v);
        else
          v = cjmadd(u[d * 3 + c], h[hs * 3 + d], v);
      }
      t[hs * 3 + c] = v;
    }
  }
  if constexpr (P == WD_F16) {
    if (MU == 3 && flip) sc = -sc;
    expand_add<MU, S, false>(acc, t, sc);
  } else if constexpr (MU == 3) {
    expand_add<MU, S, false>(acc, t, flip ? (R)-1 : (R)1);
  } else {
    expand_add<MU, S, true>(acc, t, (R)1);
  }
}

template <int P, int RC, int MU, int S, bool FWD, typename R>
__device__ __forceinline__ void hop_mrhs(cx<R> (&acc)[12], const void* __restrict__ in, int nb,
                                         const int4* sm, int hop, int tid, const void* gauge,
                                         int region, int lcb, bool flip, int VP) {
  cx<R> u[9];
  if constexpr (MrhsStage<P, RC>::on)
    unstage_link<P, R>(u, sm, hop, tid);
  else
    load_link<P, RC, R>(u, gauge, region, lcb, VP);
  hop_with_link<P, MU, S, FWD, R>(acc, in, nb, u, flip, VP);
}

template <int P, int RC, bool DAG, bool NORM>
__global__ void __launch_bounds__(MRHS_BS) mrhs_dslash_kernel(const MrhsBatch bt,
                                                              const int* __restrict__ active,
                                                              RedScratch rs, double* norm_out) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  extern __shared__ int4 smem4[];
  __shared__ double red[MRHS_BS / 32];
  const int tid = threadIdx.x;
  constexpr int SF = DAG ? -1 : 1;
  constexpr int SB_ = -SF;

  const int nprob = bt.nprob, ntiles = bt.ntiles;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int j = 0;
    while (j + 1 < nprob && tile >= bt.p[j + 1].tile0) j++;
    const MrhsProblem& pr = bt.p[j];
    const Geom g = pr.g;
    const int cb = (tile - pr.tile0) * MRHS_BS + tid;
    const bool valid = cb < g.Vh;
    const int p = pr.parity, q = 1 - p, VP = g.Vh_pad;
    int f[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
    bool fflip = false, bflip = false;
    if (valid) {
      int x0, x1, x2, x3;
      cb_coords(cb, p, g, x0, x1, x2, x3);
      const int row = cb - (x0 >> 1);
      f[0] = row + ((x0 + 1 == g.L[0] ? 0 : x0 + 1) >> 1);
      b[0] = row + ((x0 == 0 ? g.L[0] - 1 : x0 - 1) >> 1);
      f[1] = x1 == g.L[1] - 1 ? cb - (g.L[1] - 1) * g.S1 : cb + g.S1;
      b[1] = x1 == 0 ? cb + (g.L[1] - 1) * g.S1 : cb - g.S1;
      f[2] = x2 == g.L[2] - 1 ? cb - (g.L[2] - 1) * g.S2 : cb + g.S2;
      b[2] = x2 == 0 ? cb + (g.L[2] - 1) * g.S2 : cb - g.S2;
      f[3] = x3 == g.L[3] - 1 ? cb - (g.L[3] - 1) * g.S3 : cb + g.S3;
      b[3] = x3 == 0 ? cb + (g.L[3] - 1) * g.S3 : cb - g.S3;
      fflip = x3 == g.L[3] - 1;
      bflip = x3 == 0;
    }
    __syncthreads();  // the previous tile's staged links are no longer read
    if constexpr (MrhsStage<P, RC>::on) {
      if (valid) {
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
          stage_link<P, RC>(smem4, 2 * mu, tid, pr.gauge, 2 * mu + p, cb, VP);
          stage_link<P, RC>(smem4, 2 * mu + 1, tid, pr.gauge, 2 * mu + q, b[mu], VP);
        }
      }
    }
    // each thread reads back only the slots it wrote: no barrier needed here

    for (int r = 0; r < pr.nrhs; r++) {
      const bool act = active == nullptr || active[pr.rhs0 + r] != 0;
      if (!act) continue;  // uniform over the CTA
      double nrm = 0.0;
      if (valid) {
        const void* in = (const char*)pr.in + (size_t)r * pr.s_in;
        cx<R> acc[12];
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);
        const void* ga = pr.gauge;
        hop_mrhs<P, RC, 0, SF, true>(acc, in, f[0], smem4, 0, tid, ga, 0 + p, cb, false, VP);
        hop_mrhs<P, RC, 0, SB_, false>(acc, in, b[0], smem4, 1, tid, ga, 0 + q, b[0], false, VP);
        hop_mrhs<P, RC, 1, SF, true>(acc, in, f[1], smem4, 2, tid, ga, 2 + p, cb, false, VP);
        hop_mrhs<P, RC, 1, SB_, false>(acc, in, b[1], smem4, 3, tid, ga, 2 + q, b[1], false, VP);
        hop_mrhs<P, RC, 2, SF, true>(acc, in, f[2], smem4, 4, tid, ga, 4 + p, cb, false, VP);
        hop_mrhs<P, RC, 2, SB_, false>(acc, in, b[2], smem4, 5, tid, ga, 4 + q, b[2], false, VP);
        hop_mrhs<P, RC, 3, SF, true>(acc, in, f[3], smem4, 6, tid, ga, 6 + p, cb, fflip, VP);
        hop_mrhs<P, RC, 3, SB_, false>(acc, in, b[3], smem4, 7, tid, ga, 6 + q, b[3], bflip, VP);
        const R ca = (R)pr.a;
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = ca * acc[k];
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
        void* out = (char*)pr.out + (size_t)r * pr.s_out;
        store_spinor<P, R>(out, cb, VP, acc);
        if constexpr (NORM) {
          if constexpr (P == WD_F16) {
            cx<R> v[12];
            load_spinor_rw<P, R>(v, out, cb, VP);
            nrm = site_norm2(v);
          } else {
            nrm = site_norm2(acc);
          }
        }
      }
      if constexpr (NORM) {
        double v[1] = {nrm};
        block_sum<1, MRHS_BS>(v, red);
        if (tid == 0) rs.partials[(size_t)tile * MRHS_MAX + r] = v[0];
      }
    }
  }

  if constexpr (NORM) {
    // the last CTA to finish sums each right-hand side's tiles in tile order
    __shared__ bool last;
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      unsigned t = atomicAdd(rs.counter, 1u);
      last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int jj = 0; jj < nprob; jj++) {
      const MrhsProblem& pr = bt.p[jj];
      for (int r = 0; r < pr.nrhs; r++) {
        if (active != nullptr && active[pr.rhs0 + r] == 0) continue;
        double v[1] = {0.0};
        for (int t = tid; t < pr.ntiles; t += MRHS_BS)
          v[0] += __ldcg(rs.partials + (size_t)(pr.tile0 + t) * MRHS_MAX + r);
        block_sum<1, MRHS_BS>(v, red);
        if (tid == 0) norm_out[pr.rhs0 + r] = v[0];
      }
    }
    if (tid == 0) *rs.counter = 0u;
  }
}

template <int P, int RC, bool DG, bool NM>
cudaError_t launch_mrhs_one(const MrhsBatch& bt, const int* active, RedScratch rs,
                            double* norm_out, int grid, cudaStream_t st) {
  constexpr size_t smem = (size_t)MRHS_BS * MrhsStage<P, RC>::bytes_per_thread;
  static bool attr = false;  // raise the dynamic shared-memory limit once
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mrhs_dslash_kernel<P, RC, DG, NM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  mrhs_dslash_kernel<P, RC, DG, NM><<<grid, MRHS_BS, smem, st>>>(bt, active, rs, norm_out);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_mrhs_prec(const MrhsBatch& bt, int recon, bool dagger, const int* active,
                             RedScratch rs, double* norm_out, int grid, cudaStream_t st) {
  const bool nm = norm_out != nullptr;
  if (recon == 12) {
    if (dagger) return nm ? launch_mrhs_one<P, 12, true, true>(bt, active, rs, norm_out, grid, st)
                          : launch_mrhs_one<P, 12, true, false>(bt, active, rs, norm_out, grid, st);
    return nm ? launch_mrhs_one<P, 12, false, true>(bt, active, rs, norm_out, grid, st)
              : launch_mrhs_one<P, 12, false, false>(bt, active, rs, norm_out, grid, st);
  }
  if constexpr (P != WD_F16) {
    if (recon == 18) {
      if (dagger) return nm ? launch_mrhs_one<P, 18, true, true>(bt, active, rs, norm_out, grid, st)
                            : launch_mrhs_one<P, 18, true, false>(bt, active, rs, norm_out, grid, st);
      return nm ? launch_mrhs_one<P, 18, false, true>(bt, active, rs, norm_out, grid, st)
                : launch_mrhs_one<P, 18, false, false>(bt, active, rs, norm_out, grid, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace wd
