// The parity-restricted Wilson hopping kernel ("Dslash" of the paper, section
// "Wilson inverter: Main features"): one thread per output site of parity p,
//
//   out(x) = a * sum_mu [ (1 - s gamma_mu) U_mu(x) in(x+mu)
//                       + (1 + s gamma_mu) U_mu(x-mu)^+ in(x-mu) ]  + bx x(x) + cy y(x)
//
// s = +1 for H, s = -1 for H^+.  Per hop: load the neighbour spinor, project
// it to a two-spin half spinor (the projector has rank 2; paper, section
// "Local storage constraints"), multiply by the link (rows 0 and 1 loaded,
// row 2 rebuilt for 12-real storage), expand back to four spins and add.
// The antiperiodic time boundary is applied by negating the half spinor of
// hops that cross t = L3-1 <-> 0; links are never modified.
#pragma once

#include <type_traits>

#include "wd_internal.h"

namespace wd {

// Spin projection for direction MU with projector (1 - S gamma_MU) in the
// chiral basis.  psi index = spin*3 + colour, h index = half-spin*3 + colour.
template <int S, typename R>
__device__ __forceinline__ cx<R> addS(cx<R> a, cx<R> b) {
  return S > 0 ? a + b : a - b;
}

template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cx<R> (&p)[12], cx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    if constexpr (MU == 0) {          // h0 = p0 + S i p3 ; h1 = p1 + S i p2
      h[c] = addS<S>(p[c], ti(p[9 + c]));
      h[3 + c] = addS<S>(p[3 + c], ti(p[6 + c]));
    } else if constexpr (MU == 1) {   // h0 = p0 + S p3 ; h1 = p1 - S p2
      h[c] = addS<S>(p[c], p[9 + c]);
      h[3 + c] = addS<-S>(p[3 + c], p[6 + c]);
    } else if constexpr (MU == 2) {   // h0 = p0 + S i p2 ; h1 = p1 - S i p3
      h[c] = addS<S>(p[c], ti(p[6 + c]));
      h[3 + c] = addS<-S>(p[3 + c], ti(p[9 + c]));
    } else {                          // h0 = p0 - S p2 ; h1 = p1 - S p3
      h[c] = addS<-S>(p[c], p[6 + c]);
      h[3 + c] = addS<-S>(p[3 + c], p[9 + c]);
    }
  }
}

// Expansion of the transported half spinor t back to four spins, added to acc.
template <int MU, int S, typename R>
__device__ __forceinline__ void expand_add(cx<R> (&acc)[12], const cx<R> (&t)[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = acc[c] + t[c];
    acc[3 + c] = acc[3 + c] + t[3 + c];
    if constexpr (MU == 0) {          // lower = (-S i t1, -S i t0)
      acc[6 + c] = addS<-S>(acc[6 + c], ti(t[3 + c]));
      acc[9 + c] = addS<-S>(acc[9 + c], ti(t[c]));
    } else if constexpr (MU == 1) {   // lower = (-S t1, S t0)
      acc[6 + c] = addS<-S>(acc[6 + c], t[3 + c]);
      acc[9 + c] = addS<S>(acc[9 + c], t[c]);
    } else if constexpr (MU == 2) {   // lower = (-S i t0, S i t1)
      acc[6 + c] = addS<-S>(acc[6 + c], ti(t[c]));
      acc[9 + c] = addS<S>(acc[9 + c], ti(t[3 + c]));
    } else {                          // lower = (-S t0, -S t1)
      acc[6 + c] = addS<-S>(acc[6 + c], t[c]);
      acc[9 + c] = addS<-S>(acc[9 + c], t[3 + c]);
    }
  }
}

// One hop: neighbour site nb (opposite parity), link in `region` at site lcb.
// FWD: U h ; backward: U^+ h.  flip: negate (antiperiodic crossing).
template <int P, int RC, int MU, int S, bool FWD, typename R>
__device__ __forceinline__ void hop(cx<R> (&acc)[12], const void* __restrict__ in,
                                    const void* __restrict__ gauge, int nb, int region, int lcb,
                                    bool flip, int Vh_pad) {
  cx<R> psi[12];
  load_spinor<P, R>(psi, in, nb, Vh_pad);
  cx<R> u[9];
  load_link<P, RC, R>(u, gauge, region, lcb, Vh_pad);
  cx<R> h[6];
  project<MU, S>(psi, h);
  if (MU == 3 && flip) {
#pragma unroll
    for (int k = 0; k < 6; k++) h[k] = mk<R>(-h[k].r, -h[k].i);
  }
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
  expand_add<MU, S>(acc, t);
}

template <int P, int RC, bool DAG, bool NORM, int BS>
__global__ void __launch_bounds__(BS) dslash_kernel(const DslashArgs a) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  const Geom& g = a.g;
  const int cb = blockIdx.x * BS + threadIdx.x;
  double nrm = 0.0;
  if (cb < g.Vh) {
    const int p = a.parity;
    const int xh = cb % g.Lh0;
    int r = cb / g.Lh0;
    const int x1 = r % g.L[1];
    r /= g.L[1];
    const int x2 = r % g.L[2];
    const int x3 = r / g.L[2];
    const int x0 = 2 * xh + ((p + x1 + x2 + x3) & 1);
    const int row = cb - xh;

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

    // forward hops use (1 - s gamma), backward (1 + s gamma)
    constexpr int SF = DAG ? -1 : 1;
    constexpr int SB_ = -SF;
    const int q = 1 - p;
    const int VP = g.Vh_pad;

    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);

    hop<P, RC, 0, SF, true>(acc, a.in, a.gauge, f0, 0 + p, cb, false, VP);
    hop<P, RC, 0, SB_, false>(acc, a.in, a.gauge, b0, 0 + q, b0, false, VP);
    hop<P, RC, 1, SF, true>(acc, a.in, a.gauge, f1, 2 + p, cb, false, VP);
    hop<P, RC, 1, SB_, false>(acc, a.in, a.gauge, b1, 2 + q, b1, false, VP);
    hop<P, RC, 2, SF, true>(acc, a.in, a.gauge, f2, 4 + p, cb, false, VP);
    hop<P, RC, 2, SB_, false>(acc, a.in, a.gauge, b2, 4 + q, b2, false, VP);
    hop<P, RC, 3, SF, true>(acc, a.in, a.gauge, f3, 6 + p, cb, fflip, VP);
    hop<P, RC, 3, SB_, false>(acc, a.in, a.gauge, b3, 6 + q, b3, bflip, VP);

    const R ca = (R)a.a;
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = ca * acc[k];
    if (a.x) {
      cx<R> v[12];
      load_spinor_rw<P, R>(v, a.x, cb, VP);
      const R cbx = (R)a.bx;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[k].r = fma(cbx, v[k].r, acc[k].r);
        acc[k].i = fma(cbx, v[k].i, acc[k].i);
      }
    }
    if (a.y) {
      cx<R> v[12];
      load_spinor_rw<P, R>(v, a.y, cb, VP);
      const R ccy = (R)a.cy;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[k].r = fma(ccy, v[k].r, acc[k].r);
        acc[k].i = fma(ccy, v[k].i, acc[k].i);
      }
    }
    store_spinor<P, R>(a.out, cb, VP, acc);
    if constexpr (NORM) {
      if constexpr (P == WD_F16) {
        // the norm of what was stored (after rounding to half)
        cx<R> v[12];
        load_spinor_rw<P, R>(v, a.out, cb, VP);
#pragma unroll
        for (int k = 0; k < 12; k++) nrm += (double)v[k].r * v[k].r + (double)v[k].i * v[k].i;
      } else {
#pragma unroll
        for (int k = 0; k < 12; k++) nrm += (double)acc[k].r * acc[k].r + (double)acc[k].i * acc[k].i;
      }
    }
  }
  if constexpr (NORM) {
    double v[1] = {nrm};
    double tot[1];
    if (grid_reduce<1, BS>(v, a.rs, tot) && threadIdx.x == 0) *a.norm_out = tot[0];
  }
}

// Launch one instance; the .cu file of each precision instantiates it.
template <int P>
cudaError_t launch_dslash_prec(const DslashArgs& a, int recon, bool dagger, cudaStream_t st) {
  const int BS = DSLASH_BS;
  dim3 grid((a.g.Vh + BS - 1) / BS), block(BS);
  const bool norm = a.norm_out != nullptr;
#define WD_LAUNCH(RC, DG, NM) dslash_kernel<P, RC, DG, NM, DSLASH_BS><<<grid, block, 0, st>>>(a)
  if constexpr (P == WD_F16) {
    if (recon != 12) return cudaErrorInvalidValue;
    if (dagger) { if (norm) WD_LAUNCH(12, true, true); else WD_LAUNCH(12, true, false); }
    else        { if (norm) WD_LAUNCH(12, false, true); else WD_LAUNCH(12, false, false); }
  } else {
    if (recon == 12) {
      if (dagger) { if (norm) WD_LAUNCH(12, true, true); else WD_LAUNCH(12, true, false); }
      else        { if (norm) WD_LAUNCH(12, false, true); else WD_LAUNCH(12, false, false); }
    } else {
      if (dagger) { if (norm) WD_LAUNCH(18, true, true); else WD_LAUNCH(18, true, false); }
      else        { if (norm) WD_LAUNCH(18, false, true); else WD_LAUNCH(18, false, false); }
    }
  }
#undef WD_LAUNCH
  return cudaGetLastError();
}

}  // namespace wd
