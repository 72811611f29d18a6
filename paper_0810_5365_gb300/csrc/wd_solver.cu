// Even-odd preconditioned, mixed-precision CG solver for D x = b.
//
// The paper's inverter is an even-odd preconditioned conjugate gradient built
// from separate kernels (Dslash, Dslash^+, an FP64 dot product and BLAS-like
// updates) with negligible host-device traffic (section "Wilson inverter:
// Main features"; performance in its Fig. 2).  This file realises it as:
//
//  * Schur complement on the even sites:
//      Mhat = 1 - kappa^2 H_eo H_oe,  bhat_e = b_e + kappa H_eo b_o,
//      x_o = b_o + kappa H_oe x_e   (then D x = b exactly on the odd rows, and
//      the even-row residual equals bhat_e - Mhat x_e);
//  * CG on the normal equations Mhat^+ Mhat x_e = Mhat^+ bhat_e in the CGLS
//    arrangement, which tracks r = bhat - Mhat x itself;
//  * inner ("sloppy") iterations in FP32 or FP16 with FP64 reliable updates
//    (Sleijpen and van der Vorst, Computing 56, 1996): every
//    `reliable_interval` iterations, and whenever the sloppy residual looks
//    converged, the sloppy solution is folded into an FP64 accumulator and
//    the true residual is recomputed with the FP64 operator;
//  * all CG scalars stay on the device; each block of `check_interval`
//    iterations is one captured CUDA graph; the host reads four doubles per
//    block to decide on convergence;
//  * the norms and dot products are fused into the kernels that produce the
//    vectors (per-CTA partials, summed in a fixed order by a one-CTA launch
//    behind them), and consecutive launches overlap (programmatic dependent
//    launch).
#include <chrono>
#include <cmath>
#include <cstring>

#include "wd_internal.h"

namespace wd {

struct CgScalars {
  double gamma[2];  // ||s||^2, ping-pong between consecutive iterations
  double qq;        // ||q||^2, q = Mhat p
  double rr;        // ||r||^2 of the sloppy residual
  double r64;       // ||bhat - Mhat x64||^2 (FP64)
  double bnorm2;    // ||b||^2 of the full right-hand side
  double res_e, res_o;  // ||b - D x||^2 on even / odd sites
  // BiCGstab (complex scalars as (re, im), ping-pong between iterations)
  double rho[2][2];  // <r0, r>
  double rv[2][2];   // <r0, v>
  double tts[2][3];  // ||t||^2, <t, s>
};

__host__ __device__ __forceinline__ void zdiv(double ar, double ai, double br, double bi,
                                              double& cr, double& ci) {
  const double d = br * br + bi * bi;
  cr = (ar * br + ai * bi) / d;
  ci = (ai * br - ar * bi) / d;
}

// One site of a packed field as it sits in memory (the format load_spinor_rw
// reads), so that a kernel can issue the loads of its next site before it
// computes the current one.
template <int P>
struct RawSite;
template <>
struct RawSite<WD_F16> {
  int4 v[3];
  float s;
};
template <>
struct RawSite<WD_F32> {
  float4 v[6];
};
template <>
struct RawSite<WD_F64> {
  double2 v[12];
};

template <int P>
__device__ __forceinline__ void load_raw(RawSite<P>& o, const void* base, int cb, int Vh_pad) {
  if constexpr (P == WD_F16) {
    const int4* p = (const int4*)base;
#pragma unroll
    for (int k = 0; k < 3; k++) o.v[k] = p[sbi(cb, k, 3)];
    o.s = ((const float*)((const char*)base + (size_t)Vh_pad * 48))[cb];
  } else if constexpr (P == WD_F32) {
    const float4* p = (const float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++) o.v[k] = p[sbi(cb, k, 6)];
  } else {
    const double2* p = (const double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) o.v[k] = p[sbi(cb, k, 12)];
  }
}

// the values of a raw site, with the arithmetic of load_spinor_rw
template <int P, typename R>
__device__ __forceinline__ void unpack_raw(cx<R> (&s)[12], const RawSite<P>& o) {
  if constexpr (P == WD_F16) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const __half2* h = reinterpret_cast<const __half2*>(&o.v[k]);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 f = __half22float2(h[j]);
        s[4 * k + j] = mk<R>((R)(f.x * o.s), (R)(f.y * o.s));
      }
    }
  } else if constexpr (P == WD_F32) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      s[2 * k] = mk<R>((R)o.v[k].x, (R)o.v[k].y);
      s[2 * k + 1] = mk<R>((R)o.v[k].z, (R)o.v[k].w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) s[k] = mk<R>((R)o.v[k].x, (R)o.v[k].y);
  }
}

// The CG vector updates (and BiCGstab's p and s updates below) stream a few
// fields once, about 10-20 us per call on 24^3x48.  They run on a grid of resident CTAs only (update_grid)
// and each thread loads its next site before it computes the current one,
// so that the load latency is paid about once per thread instead of once
// per CTA generation.

// r -= alpha q ; rr = ||r||^2 ; alpha = gamma[kp] / qq
template <int P, int BS>
__global__ void __launch_bounds__(BS) cg_update_r(char* r, const char* __restrict__ q,
                                                  CgScalars* sc, int kp, Geom g, RedScratch rs) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  pdl_begin();
  const R alpha = (R)(sc->gamma[kp] / sc->qq);
  R acc[1] = {(R)0};
  const int stride = gridDim.x * BS, VP = g.Vh_pad;
  int cb = blockIdx.x * BS + threadIdx.x;
  RawSite<P> ra, rb;
  if (cb < g.Vh) {
    load_raw<P>(ra, r, cb, VP);
    load_raw<P>(rb, q, cb, VP);
  }
  for (; cb < g.Vh; cb += stride) {
    const int nx = cb + stride;
    RawSite<P> na, nb;
    if (nx < g.Vh) {
      load_raw<P>(na, r, nx, VP);
      load_raw<P>(nb, q, nx, VP);
    }
    cx<R> a[12], b[12];
    unpack_raw<P, R>(a, ra);
    unpack_raw<P, R>(b, rb);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      a[k].r = fma(-alpha, b[k].r, a[k].r);
      a[k].i = fma(-alpha, b[k].i, a[k].i);
    }
    store_spinor<P, R>(r, cb, VP, a);
    acc[0] += site_norm2<R>(a);
    ra = na;
    rb = nb;
  }
  block_partials<1, BS>(acc, rs.partials);  // summed into sc->rr by the next launch
}

// x += alpha p ; p = s + beta p ; beta = gamma[1-kp] / gamma[kp]
template <int P, int PX, int BS>
__global__ void __launch_bounds__(BS, (P == WD_F16 ? 2 : 1))
    cg_update_xp(char* x, char* p, const char* __restrict__ s, const CgScalars* sc, int kp,
                 Geom g) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  using RX = typename std::conditional<PX == WD_F64, double, float>::type;
  pdl_begin();
  const double g0 = sc->gamma[kp];
  const RX alpha = (RX)(g0 / sc->qq);
  const R beta = (R)(sc->gamma[1 - kp] / g0);
  const int stride = gridDim.x * BS, VP = g.Vh_pad;
  int cb = blockIdx.x * BS + threadIdx.x;
  RawSite<P> rp, rsv;
  RawSite<PX> rx;
  if (cb < g.Vh) {
    load_raw<P>(rp, p, cb, VP);
    load_raw<P>(rsv, s, cb, VP);
    load_raw<PX>(rx, x, cb, VP);
  }
  for (; cb < g.Vh; cb += stride) {
    const int nx = cb + stride;
    RawSite<P> np, ns;
    RawSite<PX> nxr;
    if (nx < g.Vh) {
      load_raw<P>(np, p, nx, VP);
      load_raw<P>(ns, s, nx, VP);
      load_raw<PX>(nxr, x, nx, VP);
    }
    cx<R> pv[12], sv[12];
    cx<RX> xv[12];
    unpack_raw<P, R>(pv, rp);
    unpack_raw<P, R>(sv, rsv);
    unpack_raw<PX, RX>(xv, rx);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      xv[k].r = fma(alpha, (RX)pv[k].r, xv[k].r);
      xv[k].i = fma(alpha, (RX)pv[k].i, xv[k].i);
      pv[k].r = fma(beta, pv[k].r, sv[k].r);
      pv[k].i = fma(beta, pv[k].i, sv[k].i);
    }
    store_spinor<PX, RX>(x, cb, VP, xv);
    store_spinor<P, R>(p, cb, VP, pv);
    rp = np;
    rsv = ns;
    rx = nxr;
  }
}

// The grid of an update kernel: as many CTAs of 256 threads as are resident
// at once (the occupancy query), at most one per 256 sites.
template <typename K>
static int resident_grid(K kernel, int vh) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long need = (vh + 255) / 256;
  const long long cap = (long long)per_sm * num_sms();
  return (int)(need < cap ? need : cap);
}


// x64 += xs ; xs = 0
template <int PX, int BS>
__global__ void __launch_bounds__(BS) ru_accumulate(char* x64, char* xs, Geom g) {
  using RX = typename std::conditional<PX == WD_F64, double, float>::type;
  for (int cb = blockIdx.x * BS + threadIdx.x; cb < g.Vh; cb += gridDim.x * BS) {
    cx<double> a[12];
    cx<RX> b[12];
    load_spinor_rw<WD_F64, double>(a, x64, cb, g.Vh_pad);
    load_spinor_rw<PX, RX>(b, xs, cb, g.Vh_pad);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      a[k].r += (double)b[k].r;
      a[k].i += (double)b[k].i;
      b[k] = mk<RX>(0, 0);
    }
    store_spinor<WD_F64, double>(x64, cb, g.Vh_pad, a);
    store_spinor<PX, RX>(xs, cb, g.Vh_pad, b);
  }
}

// ---------------------------------------------------------------------------
// BiCGstab updates (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) on
// the Schur operator; the paper reports a BiCGstab inverter beside its CG
// (section "Performance").  Scalars are recomputed by every thread from the
// reductions in CgScalars; kp selects the current slot.
// ---------------------------------------------------------------------------

// p = r + beta (p - omega_old v),  beta = (rho_new / rho_old) (alpha_old / omega_old)
template <int P, int BS>
__global__ void __launch_bounds__(BS) bicg_update_p(char* p, const char* __restrict__ r,
                                                    const char* __restrict__ v,
                                                    const CgScalars* sc, int kp, Geom g) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  pdl_begin();
  const int kq = 1 - kp;
  double ar, ai, wr, wi, t1r, t1i, t2r, t2i, br, bi;
  zdiv(sc->rho[kq][0], sc->rho[kq][1], sc->rv[kq][0], sc->rv[kq][1], ar, ai);   // alpha_old
  zdiv(sc->tts[kq][1], sc->tts[kq][2], sc->tts[kq][0], 0.0, wr, wi);          // omega_old
  zdiv(sc->rho[kp][0], sc->rho[kp][1], sc->rho[kq][0], sc->rho[kq][1], t1r, t1i);
  zdiv(ar, ai, wr, wi, t2r, t2i);
  br = t1r * t2r - t1i * t2i;
  bi = t1r * t2i + t1i * t2r;
  const R Br = (R)br, Bi = (R)bi, Wr = (R)wr, Wi = (R)wi;
  // resident grid, next site's loads first (as in cg_update_xp)
  const int stride = gridDim.x * BS, VP = g.Vh_pad;
  int cb = blockIdx.x * BS + threadIdx.x;
  RawSite<P> rp, rr, rv;
  if (cb < g.Vh) {
    load_raw<P>(rp, p, cb, VP);
    load_raw<P>(rr, r, cb, VP);
    load_raw<P>(rv, v, cb, VP);
  }
  for (; cb < g.Vh; cb += stride) {
    const int nx = cb + stride;
    RawSite<P> np, nr, nv;
    if (nx < g.Vh) {
      load_raw<P>(np, p, nx, VP);
      load_raw<P>(nr, r, nx, VP);
      load_raw<P>(nv, v, nx, VP);
    }
    cx<R> pv[12], rv_[12], vv[12];
    unpack_raw<P, R>(pv, rp);
    unpack_raw<P, R>(rv_, rr);
    unpack_raw<P, R>(vv, rv);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      // u = p - omega v
      const R ur = pv[k].r - (Wr * vv[k].r - Wi * vv[k].i);
      const R ui = pv[k].i - (Wr * vv[k].i + Wi * vv[k].r);
      pv[k].r = rv_[k].r + (Br * ur - Bi * ui);
      pv[k].i = rv_[k].i + (Br * ui + Bi * ur);
    }
    store_spinor<P, R>(p, cb, VP, pv);
    rp = np;
    rr = nr;
    rv = nv;
  }
}

// s = r - alpha v,  alpha = rho / <r0, v>
template <int P, int BS>
__global__ void __launch_bounds__(BS) bicg_update_s(char* s, const char* __restrict__ r,
                                                    const char* __restrict__ v,
                                                    const CgScalars* sc, int kp, Geom g) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  pdl_begin();
  double ar, ai;
  zdiv(sc->rho[kp][0], sc->rho[kp][1], sc->rv[kp][0], sc->rv[kp][1], ar, ai);
  const R Ar = (R)ar, Ai = (R)ai;
  // resident grid, next site's loads first (as in cg_update_r)
  const int stride = gridDim.x * BS, VP = g.Vh_pad;
  int cb = blockIdx.x * BS + threadIdx.x;
  RawSite<P> rr, rv;
  if (cb < g.Vh) {
    load_raw<P>(rr, r, cb, VP);
    load_raw<P>(rv, v, cb, VP);
  }
  for (; cb < g.Vh; cb += stride) {
    const int nx = cb + stride;
    RawSite<P> nr, nv;
    if (nx < g.Vh) {
      load_raw<P>(nr, r, nx, VP);
      load_raw<P>(nv, v, nx, VP);
    }
    cx<R> rv_[12], vv[12];
    unpack_raw<P, R>(rv_, rr);
    unpack_raw<P, R>(vv, rv);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      rv_[k].r -= Ar * vv[k].r - Ai * vv[k].i;
      rv_[k].i -= Ar * vv[k].i + Ai * vv[k].r;
    }
    store_spinor<P, R>(s, cb, VP, rv_);
    rr = nr;
    rv = nv;
  }
}

// x += alpha p + omega s ; r = s - omega t ; rho_next = <r0, r> ; rr = ||r||^2
template <int P, int PX, int BS>
__global__ void __launch_bounds__(BS) bicg_update_xr(char* x, char* r, const char* __restrict__ p,
                                                     const char* __restrict__ s,
                                                     const char* __restrict__ t,
                                                     const char* __restrict__ r0, CgScalars* sc,
                                                     int kp, Geom g, RedScratch rs) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  using RX = typename std::conditional<PX == WD_F64, double, float>::type;
  pdl_begin();
  double ar, ai, wr, wi;
  zdiv(sc->rho[kp][0], sc->rho[kp][1], sc->rv[kp][0], sc->rv[kp][1], ar, ai);
  zdiv(sc->tts[kp][1], sc->tts[kp][2], sc->tts[kp][0], 0.0, wr, wi);
  const RX Ar = (RX)ar, Ai = (RX)ai, Wxr = (RX)wr, Wxi = (RX)wi;
  const R Wr = (R)wr, Wi = (R)wi;
  R acc[3] = {(R)0, (R)0, (R)0};
  if constexpr (P == WD_F64) {
    // (FP64: five prefetched sites do not fit the register file; plain loop)
    for (int cb = blockIdx.x * BS + threadIdx.x; cb < g.Vh; cb += gridDim.x * BS) {
      cx<R> pv[12], sv[12], tv[12], zv[12];
      cx<RX> xv[12];
      load_spinor_rw<P, R>(pv, p, cb, g.Vh_pad);
      load_spinor_rw<P, R>(sv, s, cb, g.Vh_pad);
      load_spinor_rw<P, R>(tv, t, cb, g.Vh_pad);
      load_spinor_rw<PX, RX>(xv, x, cb, g.Vh_pad);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const RX pr = (RX)pv[k].r, pi = (RX)pv[k].i, sr = (RX)sv[k].r, si = (RX)sv[k].i;
        xv[k].r += Ar * pr - Ai * pi + Wxr * sr - Wxi * si;
        xv[k].i += Ar * pi + Ai * pr + Wxr * si + Wxi * sr;
        sv[k].r -= Wr * tv[k].r - Wi * tv[k].i;
        sv[k].i -= Wr * tv[k].i + Wi * tv[k].r;
      }
      store_spinor<PX, RX>(x, cb, g.Vh_pad, xv);
      store_spinor<P, R>(r, cb, g.Vh_pad, sv);
      load_spinor_rw<P, R>(zv, r0, cb, g.Vh_pad);
      site_cdot(zv, sv, acc[0], acc[1]);
      acc[2] += site_norm2<R>(sv);
    }
  } else {
    // resident grid, next site's loads first (as in cg_update_xp)
    const int stride = gridDim.x * BS, VP = g.Vh_pad;
    int cb = blockIdx.x * BS + threadIdx.x;
    RawSite<P> rp, rsv, rt, rz;
    RawSite<PX> rx;
    if (cb < g.Vh) {
      load_raw<P>(rp, p, cb, VP);
      load_raw<P>(rsv, s, cb, VP);
      load_raw<P>(rt, t, cb, VP);
      load_raw<PX>(rx, x, cb, VP);
      load_raw<P>(rz, r0, cb, VP);
    }
    for (; cb < g.Vh; cb += stride) {
      const int nx = cb + stride;
      RawSite<P> np, ns, nt, nz;
      RawSite<PX> nxr;
      if (nx < g.Vh) {
        load_raw<P>(np, p, nx, VP);
        load_raw<P>(ns, s, nx, VP);
        load_raw<P>(nt, t, nx, VP);
        load_raw<PX>(nxr, x, nx, VP);
        load_raw<P>(nz, r0, nx, VP);
      }
      cx<R> pv[12], sv[12], tv[12], zv[12];
      cx<RX> xv[12];
      unpack_raw<P, R>(pv, rp);
      unpack_raw<P, R>(sv, rsv);
      unpack_raw<P, R>(tv, rt);
      unpack_raw<PX, RX>(xv, rx);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const RX pr = (RX)pv[k].r, pi = (RX)pv[k].i, sr = (RX)sv[k].r, si = (RX)sv[k].i;
        xv[k].r += Ar * pr - Ai * pi + Wxr * sr - Wxi * si;
        xv[k].i += Ar * pi + Ai * pr + Wxr * si + Wxi * sr;
        sv[k].r -= Wr * tv[k].r - Wi * tv[k].i;
        sv[k].i -= Wr * tv[k].i + Wi * tv[k].r;
      }
      store_spinor<PX, RX>(x, cb, VP, xv);
      // (FP16: sv becomes the site as stored, the values load_spinor_rw would
      // read back)
      if constexpr (P == WD_F16)
        store_spinor_f16<R, true>(r, cb, VP, sv);
      else
        store_spinor<P, R>(r, cb, VP, sv);
      unpack_raw<P, R>(zv, rz);
      site_cdot(zv, sv, acc[0], acc[1]);
      acc[2] += site_norm2<R>(sv);
      rp = np;
      rsv = ns;
      rt = nt;
      rx = nxr;
      rz = nz;
    }
  }
  // summed into rho[1 - kp] and rr by the next launch
  block_partials<3, BS>(acc, rs.partials);
}

// restart: rho[0] = ||r||^2 (r0 = r), and the "previous" slot set so that the
// first p-update gives p = r (p = v = 0 beforehand)
__global__ void bicg_restart_scalars(CgScalars* sc) {
  sc->rho[0][0] = sc->rr;
  sc->rho[0][1] = 0.0;
  sc->rho[1][0] = 1.0;
  sc->rho[1][1] = 0.0;
  sc->rv[1][0] = 1.0;
  sc->rv[1][1] = 0.0;
  sc->tts[1][0] = 1.0;
  sc->tts[1][1] = 1.0;
  sc->tts[1][2] = 0.0;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

template <int P, int PX>
static void update_grids_t(int vh, int (&grid)[5]) {
  grid[0] = resident_grid(cg_update_r<P, 256>, vh);
  grid[1] = resident_grid(cg_update_xp<P, PX, 256>, vh);
  grid[2] = resident_grid(bicg_update_p<P, 256>, vh);
  grid[3] = resident_grid(bicg_update_s<P, 256>, vh);
  grid[4] = resident_grid(bicg_update_xr<P, PX, 256>, vh);
}

struct Workspace {
  int dims[4] = {0, 0, 0, 0};
  int sprec = -1, srecon = 0, orecon = 0;
  Geom g{};
  void* g64 = nullptr;   // FP64 gauge (outer_recon)
  void* gs = nullptr;    // sloppy gauge (may alias g64)
  void* b64 = nullptr;   // full FP64 rhs (even half, odd half)
  void* x64 = nullptr;   // full FP64 solution
  void* rf64 = nullptr;  // full FP64 residual b - D x
  void* bhat = nullptr;  // even FP64
  void* r64 = nullptr;   // even FP64
  void* t64 = nullptr;   // odd FP64 temporary
  void* p = nullptr;     // sloppy even fields
  void* q = nullptr;
  void* r = nullptr;
  void* s = nullptr;
  void* ts = nullptr;    // sloppy odd temporary
  void* t = nullptr;     // sloppy even (BiCGstab: t = A s)
  void* r0 = nullptr;    // sloppy even (BiCGstab shadow residual)
  void* xs = nullptr;    // sloppy solution accumulator (FP32 for FP16 inner)
  double* canon_spinor = nullptr;  // staging for host spinors
  double* canon_gauge = nullptr;   // staging for a host gauge field
  double* gf_gauge = nullptr;      // temporal-gauge links (canonical)
  double* gf_omega = nullptr;      // the gauge transformation (canonical)
  double* gf_spinor = nullptr;     // rotated right-hand side (canonical)
  CgScalars* sc = nullptr;
  CgScalars* sc_host = nullptr;    // pinned
  // grids of cg_update_r, cg_update_xp, bicg_update_p, bicg_update_s,
  // bicg_update_xr
  int upd_grid[5] = {1, 1, 1, 1, 1};
  cudaStream_t cap = nullptr;      // private capture stream
  // the instantiated iteration graph of the last solve, reused by the next
  // solve on this workspace with the same key (its kernels hold workspace
  // pointers, kappa and the reduction scratch by value)
  cudaGraphExec_t exec = nullptr;
  double ex_kappa = 0.0;
  int ex_chunk = 0, ex_tg = -1, ex_bicg = -1;
  const void* ex_partials = nullptr;
  const void* ex_counter = nullptr;
};

static Workspace& ws() {
  static Workspace w;
  return w;
}

static void ws_free() {
  Workspace& w = ws();
  if (w.exec) cudaGraphExecDestroy(w.exec);
  w.exec = nullptr;
  void* bufs[] = {w.g64, w.b64, w.x64, w.rf64, w.bhat, w.r64, w.t64, w.p, w.q, w.r,
                  w.s, w.ts, w.t, w.r0, w.xs, w.canon_spinor, w.canon_gauge, w.sc,
                  w.gf_gauge, w.gf_omega, w.gf_spinor};
  if (w.gs && w.gs != w.g64) cudaFree(w.gs);
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (w.sc_host) cudaFreeHost(w.sc_host);
  if (w.cap) cudaStreamDestroy(w.cap);
  w = Workspace();
}

void solver_finalize() { ws_free(); }

static int sloppy_x_prec(int sprec) { return sprec == WD_F64 ? WD_F64 : WD_F32; }

#define WD_CK(call)                                        \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) {                               \
      state().last_cuda_error = (int)e_;                   \
      return WD_ERR_CUDA;                                  \
    }                                                      \
  } while (0)

static int ws_ensure(const int dims[4], int sprec, int srecon, int orecon) {
  Workspace& w = ws();
  if (w.sc && std::memcmp(w.dims, dims, sizeof(w.dims)) == 0 && w.sprec == sprec &&
      w.srecon == srecon && w.orecon == orecon)
    return WD_OK;
  cudaDeviceSynchronize();
  ws_free();
  Geom g = make_geom(dims);
  std::memcpy(w.dims, dims, sizeof(w.dims));
  w.sprec = sprec;
  w.srecon = srecon;
  w.orecon = orecon;
  w.g = g;
  size_t h64 = spinor_half_bytes(g, WD_F64), hs = spinor_half_bytes(g, sprec);
  size_t hx = spinor_half_bytes(g, sloppy_x_prec(sprec));
  WD_CK(cudaMalloc(&w.g64, gauge_bytes(g, WD_F64, orecon)));
  if (sprec == WD_F64 && srecon == orecon)
    w.gs = w.g64;
  else
    WD_CK(cudaMalloc(&w.gs, gauge_bytes(g, sprec, srecon)));
  WD_CK(cudaMalloc(&w.b64, 2 * h64));
  WD_CK(cudaMalloc(&w.x64, 2 * h64));
  WD_CK(cudaMalloc(&w.rf64, 2 * h64));
  WD_CK(cudaMalloc(&w.bhat, h64));
  WD_CK(cudaMalloc(&w.r64, h64));
  WD_CK(cudaMalloc(&w.t64, h64));
  WD_CK(cudaMalloc(&w.p, hs));
  WD_CK(cudaMalloc(&w.q, hs));
  WD_CK(cudaMalloc(&w.r, hs));
  WD_CK(cudaMalloc(&w.s, hs));
  WD_CK(cudaMalloc(&w.ts, hs));
  WD_CK(cudaMalloc(&w.t, hs));
  WD_CK(cudaMalloc(&w.r0, hs));
  WD_CK(cudaMalloc(&w.xs, hx));
  WD_CK(cudaMalloc(&w.sc, sizeof(CgScalars)));
  WD_CK(cudaMemset(w.sc, 0, sizeof(CgScalars)));
  WD_CK(cudaMallocHost(&w.sc_host, sizeof(CgScalars)));
  WD_CK(cudaStreamCreateWithFlags(&w.cap, cudaStreamNonBlocking));
  // the largest reduction grid used below is a dslash over Vh sites, with up
  // to three sums (BiCGstab's ||t||^2, <t, s>)
  WD_CK(ensure_scratch((size_t)((g.Vh + 127) / 128) * 3 + 1024));
  switch (sprec) {
    case WD_F64: update_grids_t<WD_F64, WD_F64>(g.Vh, w.upd_grid); break;
    case WD_F32: update_grids_t<WD_F32, WD_F32>(g.Vh, w.upd_grid); break;
    default: update_grids_t<WD_F16, WD_F32>(g.Vh, w.upd_grid); break;
  }
  return WD_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// the solve
// ---------------------------------------------------------------------------

namespace {

struct Ctx {
  Workspace* w;
  cudaStream_t st;
  double kappa;
  int sprec, srecon, orecon, xprec;
  int tg = 0;
  int bicg = 0;
  double dslash_calls = 0;
};

cudaError_t dsl(Ctx& c, int prec, int recon, const void* gauge, void* out, const void* in,
                int parity, int dagger, double a, const void* x, double bx, const void* y,
                double cy, double* norm, cudaStream_t st, int red_mode = RED_NORM,
                const void* z = nullptr) {
  DslashArgs d;
  d.out = out;
  d.in = in;
  d.gauge = gauge;
  d.x = x;
  d.y = y;
  d.a = a;
  d.bx = bx;
  d.cy = cy;
  d.norm_out = norm;
  d.rs = scratch();
  d.g = c.w->g;
  d.parity = parity;
  d.tg = c.tg;
  d.red_mode = red_mode;
  d.z = z;
  c.dslash_calls += 1;
  return launch_dslash(prec, d, recon, dagger != 0, st);
}

// q = Mhat p (sloppy), with ||q||^2 -> sc->qq
cudaError_t mhat_sloppy(Ctx& c, void* out, const void* in, int dagger, double* norm,
                        cudaStream_t st) {
  Workspace& w = *c.w;
  cudaError_t e = dsl(c, c.sprec, c.srecon, w.gs, w.ts, in, WD_ODD, dagger, 1.0, nullptr, 0,
                      nullptr, 0, nullptr, st);
  if (e != cudaSuccess) return e;
  return dsl(c, c.sprec, c.srecon, w.gs, out, w.ts, WD_EVEN, dagger, -c.kappa * c.kappa, in, 1.0,
             nullptr, 0, norm, st);
}

template <int P, int PX>
cudaError_t iteration_t(Ctx& c, int kp, cudaStream_t st) {
  Workspace& w = *c.w;
  const Geom& g = w.g;
  cudaError_t e = mhat_sloppy(c, w.q, w.p, 0, &w.sc->qq, st);
  if (e != cudaSuccess) return e;
  if ((e = launch_pdl(cg_update_r<P, 256>, dim3(w.upd_grid[0]), dim3(256), st, (char*)w.r,
                      (const char*)w.q, w.sc, kp, g, scratch())))
    return e;
  if ((e = sum_block_partials(1, scratch().partials, w.upd_grid[0], &w.sc->rr, st))) return e;
  e = mhat_sloppy(c, w.s, w.r, 1, &w.sc->gamma[1 - kp], st);
  if (e != cudaSuccess) return e;
  return launch_pdl(cg_update_xp<P, PX, 256>, dim3(w.upd_grid[1]), dim3(256), st, (char*)w.xs,
                    (char*)w.p, (const char*)w.s, (const CgScalars*)w.sc, kp, g);
}

// one BiCGstab iteration on A = Mhat (sloppy)
template <int P, int PX>
cudaError_t iteration_bicg_t(Ctx& c, int kp, cudaStream_t st) {
  Workspace& w = *c.w;
  const Geom& g = w.g;
  const double k2 = c.kappa * c.kappa;
  cudaError_t e;
  if ((e = launch_pdl(bicg_update_p<P, 256>, dim3(w.upd_grid[2]), dim3(256), st, (char*)w.p,
                      (const char*)w.r, (const char*)w.q, (const CgScalars*)w.sc, kp, g)))
    return e;
  // v = A p with <r0, v>
  if ((e = dsl(c, c.sprec, c.srecon, w.gs, w.ts, w.p, WD_ODD, 0, 1.0, nullptr, 0, nullptr, 0,
               nullptr, st)))
    return e;
  if ((e = dsl(c, c.sprec, c.srecon, w.gs, w.q, w.ts, WD_EVEN, 0, -k2, w.p, 1.0, nullptr, 0,
               &w.sc->rv[kp][0], st, RED_DOTZ, w.r0)))
    return e;
  if ((e = launch_pdl(bicg_update_s<P, 256>, dim3(w.upd_grid[3]), dim3(256), st, (char*)w.s,
                      (const char*)w.r, (const char*)w.q, (const CgScalars*)w.sc, kp, g)))
    return e;
  // t = A s with ||t||^2, <t, s>
  if ((e = dsl(c, c.sprec, c.srecon, w.gs, w.ts, w.s, WD_ODD, 0, 1.0, nullptr, 0, nullptr, 0,
               nullptr, st)))
    return e;
  if ((e = dsl(c, c.sprec, c.srecon, w.gs, w.t, w.ts, WD_EVEN, 0, -k2, w.s, 1.0, nullptr, 0,
               &w.sc->tts[kp][0], st, RED_NORM_DOTX)))
    return e;
  if ((e = launch_pdl(bicg_update_xr<P, PX, 256>, dim3(w.upd_grid[4]), dim3(256), st,
                      (char*)w.xs, (char*)w.r, (const char*)w.p, (const char*)w.s,
                      (const char*)w.t, (const char*)w.r0, w.sc, kp, g, scratch())))
    return e;
  SumOut o = {{&w.sc->rho[1 - kp][0], &w.sc->rho[1 - kp][1], &w.sc->rr}};
  return sum_block_partials(3, scratch().partials, w.upd_grid[4], o, st);
}

cudaError_t iteration(Ctx& c, int kp, cudaStream_t st) {
  if (c.bicg) {
    switch (c.sprec) {
      case WD_F64: return iteration_bicg_t<WD_F64, WD_F64>(c, kp, st);
      case WD_F32: return iteration_bicg_t<WD_F32, WD_F32>(c, kp, st);
      case WD_F16: return iteration_bicg_t<WD_F16, WD_F32>(c, kp, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (c.sprec) {
    case WD_F64: return iteration_t<WD_F64, WD_F64>(c, kp, st);
    case WD_F32: return iteration_t<WD_F32, WD_F32>(c, kp, st);
    case WD_F16: return iteration_t<WD_F16, WD_F32>(c, kp, st);
  }
  return cudaErrorInvalidValue;
}

// fold xs into x64 (even half), recompute r64 = bhat - Mhat x64 in FP64, and
// restart the sloppy recurrences: r = r64, s = Mhat^+ r, p = s, gamma[0] = ||s||^2.
// x_is_zero (a start from x = 0): r64 = bhat exactly, no FP64 operator needed.
cudaError_t reliable_update(Ctx& c, bool accumulate, cudaStream_t st, bool x_is_zero = false) {
  Workspace& w = *c.w;
  const Geom& g = w.g;
  cudaError_t e;
  if (accumulate) {
    int grid = blas_grid(g.Vh, 256);
    if (c.xprec == WD_F64)
      ru_accumulate<WD_F64, 256><<<grid, 256, 0, st>>>((char*)w.x64, (char*)w.xs, g);
    else
      ru_accumulate<WD_F32, 256><<<grid, 256, 0, st>>>((char*)w.x64, (char*)w.xs, g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (x_is_zero) {
    e = cudaMemcpyAsync(w.r64, w.bhat, spinor_half_bytes(g, WD_F64), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if ((e = norm2(&w.sc->r64, w.r64, g, WD_F64, 1, st)) != cudaSuccess) return e;
  } else {
    // t64 = H_oe x64_e ; r64 = kappa^2 H_eo t64 - x64_e + bhat
    e = dsl(c, WD_F64, c.orecon, w.g64, w.t64, w.x64, WD_ODD, 0, 1.0, nullptr, 0, nullptr, 0,
            nullptr, st);
    if (e != cudaSuccess) return e;
    e = dsl(c, WD_F64, c.orecon, w.g64, w.r64, w.t64, WD_EVEN, 0, c.kappa * c.kappa, w.x64,
            -1.0, w.bhat, 1.0, &w.sc->r64, st);
    if (e != cudaSuccess) return e;
  }
  if ((e = convert_spinor(w.r, c.sprec, w.r64, WD_F64, g, 1, st)) != cudaSuccess) return e;
  if (c.bicg) {
    // restart BiCGstab: r0 = r, p = v = 0, rho = ||r||^2
    const size_t hs = spinor_half_bytes(g, c.sprec);
    if ((e = convert_spinor(w.r0, c.sprec, w.r, c.sprec, g, 1, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.p, 0, hs, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.q, 0, hs, st)) != cudaSuccess) return e;
    if ((e = norm2(&w.sc->rr, w.r, g, c.sprec, 1, st)) != cudaSuccess) return e;
    bicg_restart_scalars<<<1, 1, 0, st>>>(w.sc);
    return cudaGetLastError();
  }
  e = mhat_sloppy(c, w.s, w.r, 1, &w.sc->gamma[0], st);
  if (e != cudaSuccess) return e;
  return convert_spinor(w.p, c.sprec, w.s, c.sprec, g, 1, st);
}

cudaError_t read_scalars(Ctx& c) {
  Workspace& w = *c.w;
  cudaError_t e = cudaMemcpyAsync(w.sc_host, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c.st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c.st);
}

}  // namespace

int solve_impl(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
               const wd_solve_params* prm, wd_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  wd_solve_params P;
  wd_solve_params_default(&P);
  if (prm) P = *prm;
  wd_solve_info I;
  std::memset(&I, 0, sizeof(I));
  if (P.inner_prec < WD_F64 || P.inner_prec > WD_F16) return WD_ERR_PREC;
  if (link_bytes(P.inner_prec, P.inner_recon) == 0 || link_bytes(WD_F64, P.outer_recon) == 0)
    return WD_ERR_PREC;
  if (!(P.tol > 0) || P.maxiter < 0 || P.reliable_interval < 1) return WD_ERR_ARG;
  int chunk = P.check_interval < 2 ? 2 : (P.check_interval & ~1);

  int rc = ws_ensure(dims, P.inner_prec, P.inner_recon, P.outer_recon);
  if (rc != WD_OK) return rc;
  Workspace& w = ws();
  const Geom& g = w.g;
  Ctx c;
  c.w = &w;
  c.st = state().stream;
  c.kappa = kappa;
  c.sprec = P.inner_prec;
  c.srecon = P.inner_recon;
  c.orecon = P.outer_recon;
  c.xprec = sloppy_x_prec(P.inner_prec);
  c.bicg = P.solver == WD_SOLVER_BICGSTAB;
  cudaStream_t st = c.st;
  const size_t V = 2 * (size_t)g.Vh;
  const size_t h64 = spinor_half_bytes(g, WD_F64);
  char* b_e = (char*)w.b64;
  char* b_o = b_e + h64;
  char* x_e = (char*)w.x64;
  char* x_o = x_e + h64;

  // ---- stage and pack the inputs ----
  const double* bdev = b;
  if (!is_device_ptr(b)) {
    if (!w.canon_spinor) WD_CK(cudaMalloc(&w.canon_spinor, V * 24 * sizeof(double)));
    WD_CK(cudaMemcpyAsync(w.canon_spinor, b, V * 24 * sizeof(double), cudaMemcpyHostToDevice, st));
    bdev = w.canon_spinor;
  }
  const double* gdev = gauge;
  if (!is_device_ptr(gauge)) {
    if (!w.canon_gauge) WD_CK(cudaMalloc(&w.canon_gauge, 4 * V * 18 * sizeof(double)));
    WD_CK(cudaMemcpyAsync(w.canon_gauge, gauge, 4 * V * 18 * sizeof(double),
                          cudaMemcpyHostToDevice, st));
    gdev = w.canon_gauge;
  }
  if (P.gauge_fix) {
    // solve D[U'] x' = omega b in temporal gauge, then x = omega^+ x'
    if (!w.gf_gauge) WD_CK(cudaMalloc(&w.gf_gauge, 4 * V * 18 * sizeof(double)));
    if (!w.gf_omega) WD_CK(cudaMalloc(&w.gf_omega, V * 18 * sizeof(double)));
    if (!w.gf_spinor) WD_CK(cudaMalloc(&w.gf_spinor, V * 24 * sizeof(double)));
    WD_CK(gauge_fix_temporal(w.gf_gauge, w.gf_omega, gdev, g, st));
    WD_CK(rotate_spinor(w.gf_spinor, bdev, w.gf_omega, g, 0, st));
    gdev = w.gf_gauge;
    bdev = w.gf_spinor;
    c.tg = 1;
  }
  WD_CK(pack_gauge(w.g64, gdev, g, WD_F64, P.outer_recon, st));
  if (w.gs != w.g64) WD_CK(pack_gauge(w.gs, gdev, g, P.inner_prec, P.inner_recon, st));
  WD_CK(pack_spinor(w.b64, bdev, g, WD_FULL, WD_F64, st));
  WD_CK(norm2(&w.sc->bnorm2, w.b64, g, WD_F64, 2, st));
  const bool x_dev = is_device_ptr(x);
  if (P.use_initial_guess) {
    const double* xdev = x;
    if (!x_dev) {
      if (!w.canon_spinor) WD_CK(cudaMalloc(&w.canon_spinor, V * 24 * sizeof(double)));
      WD_CK(cudaMemcpyAsync(w.canon_spinor, x, V * 24 * sizeof(double), cudaMemcpyHostToDevice, st));
      xdev = w.canon_spinor;
    }
    if (P.gauge_fix) {
      WD_CK(rotate_spinor(w.gf_spinor, xdev, w.gf_omega, g, 0, st));
      xdev = w.gf_spinor;
    }
    WD_CK(pack_spinor(w.x64, xdev, g, WD_FULL, WD_F64, st));
  } else {
    WD_CK(cudaMemsetAsync(w.x64, 0, 2 * h64, st));
  }
  WD_CK(cudaMemsetAsync(w.xs, 0, spinor_half_bytes(g, c.xprec), st));
  // bhat_e = b_e + kappa H_eo b_o
  WD_CK(dsl(c, WD_F64, c.orecon, w.g64, w.bhat, b_o, WD_EVEN, 0, kappa, b_e, 1.0, nullptr, 0,
            nullptr, st));
  WD_CK(reliable_update(c, false, st, !P.use_initial_guess));
  WD_CK(read_scalars(c));
  int ru = 0;
  const double bnorm = std::sqrt(w.sc_host->bnorm2);
  if (!(bnorm > 0) || !std::isfinite(bnorm)) {
    // b = 0 gives x = 0; a non-finite b is an error
    if (!std::isfinite(bnorm)) return WD_ERR_NONFINITE;
  }
  double target = P.tol * bnorm * 0.9;
  int status = WD_ERR_NOCONV;
  int iters = 0, last_ru = 0;
  int reliable_interval = P.inner_prec == WD_F64 ? 0x7fffffff : P.reliable_interval;

  WD_CK(cudaStreamSynchronize(st));
  // ---- the iteration graph ----
  cudaGraphExec_t exec = nullptr;
  const RedScratch rsk = scratch();
  if (P.use_graph && w.exec && w.ex_kappa == kappa && w.ex_chunk == chunk && w.ex_tg == c.tg &&
      w.ex_bicg == c.bicg && w.ex_partials == rsk.partials && w.ex_counter == rsk.counter) {
    exec = w.exec;  // the same workspace, parameters and scratch: reuse
  } else if (P.use_graph) {
    if (w.exec) cudaGraphExecDestroy(w.exec);
    w.exec = nullptr;
    cudaGraph_t graph = nullptr;
    WD_CK(cudaStreamBeginCapture(w.cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < chunk && ce == cudaSuccess; k++) ce = iteration(c, k & 1, w.cap);
    cudaError_t ee = cudaStreamEndCapture(w.cap, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      state().last_cuda_error = (int)(ce != cudaSuccess ? ce : ee);
      return WD_ERR_CUDA;
    }
    c.dslash_calls -= 4.0 * chunk;  // captured, not yet run
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      state().last_cuda_error = (int)ie;
      return WD_ERR_CUDA;
    }
    w.exec = exec;
    w.ex_kappa = kappa;
    w.ex_chunk = chunk;
    w.ex_tg = c.tg;
    w.ex_bicg = c.bicg;
    w.ex_partials = rsk.partials;
    w.ex_counter = rsk.counter;
  }

  auto now = [] { return std::chrono::steady_clock::now(); };
  auto secs = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
  };
  const auto t_loop = now();
  I.setup_seconds = secs(t0, t_loop);
  double t_ru = 0.0;
  double r64 = std::sqrt(w.sc_host->r64);
  bool converged = !(bnorm > 0) || r64 <= target;
  int bicg_restarts = 0;
  while (!converged) {
    const double g0 = c.bicg ? w.sc_host->rr : w.sc_host->gamma[0];
    if (!std::isfinite(w.sc_host->r64) || !std::isfinite(g0)) {
      status = WD_ERR_NONFINITE;
      break;
    }
    if (iters >= P.maxiter) break;
    if (!(g0 > 0)) {
      status = WD_ERR_BREAKDOWN;
      break;
    }
    // one block of iterations
    if (exec) {
      cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) { state().last_cuda_error = (int)e; status = WD_ERR_CUDA; break; }
      c.dslash_calls += 4.0 * chunk;
    } else {
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < chunk && e == cudaSuccess; k++) e = iteration(c, k & 1, st);
      if (e != cudaSuccess) { state().last_cuda_error = (int)e; status = WD_ERR_CUDA; break; }
    }
    iters += chunk;
    if (read_scalars(c) != cudaSuccess) { status = WD_ERR_CUDA; break; }
    const double rr = w.sc_host->rr;
    if (c.bicg) {
      // a BiCGstab breakdown (<r0, v> or ||t|| vanishing) shows up as a
      // non-finite scalar: drop the sloppy progress since the last reliable
      // update and restart from x64; give up after three restarts in a row
      const bool bad = !std::isfinite(rr) || !std::isfinite(w.sc_host->rho[0][0]) ||
                       !std::isfinite(w.sc_host->rho[1][0]);
      if (bad) {
        if (++bicg_restarts > 3) {
          status = WD_ERR_BREAKDOWN;
          break;
        }
        cudaError_t e = cudaMemsetAsync(w.xs, 0, spinor_half_bytes(g, c.xprec), st);
        if (e == cudaSuccess) e = reliable_update(c, false, st);
        if (e == cudaSuccess) e = read_scalars(c);
        if (e != cudaSuccess) { state().last_cuda_error = (int)e; status = WD_ERR_CUDA; break; }
        last_ru = iters;
        continue;
      }
      bicg_restarts = 0;
    } else {
      if (!std::isfinite(rr) || !std::isfinite(w.sc_host->gamma[0])) {
        status = WD_ERR_NONFINITE;
        break;
      }
      if (!(w.sc_host->qq > 0)) {
        status = WD_ERR_BREAKDOWN;
        break;
      }
    }
    const bool looks_done = std::sqrt(rr) <= target;
    if (looks_done || iters - last_ru >= reliable_interval || iters >= P.maxiter) {
      const auto t_a = now();
      cudaError_t e = reliable_update(c, true, st);
      if (e == cudaSuccess) e = read_scalars(c);
      t_ru += secs(t_a, now());
      if (e != cudaSuccess) { state().last_cuda_error = (int)e; status = WD_ERR_CUDA; break; }
      ru++;
      last_ru = iters;
      r64 = std::sqrt(w.sc_host->r64);
      if (!std::isfinite(r64)) { status = WD_ERR_NONFINITE; break; }
      if (r64 <= target) converged = true;
    }
  }
  const auto t_fin = now();
  I.reliable_seconds = t_ru;
  I.iterate_seconds = secs(t_loop, t_fin) - t_ru;
  if (converged) status = WD_OK;
  if (status == WD_ERR_CUDA) return status;

  // ---- reconstruct the odd sites and measure the true residual ----
  // x_o = b_o + kappa H_oe x_e
  WD_CK(dsl(c, WD_F64, c.orecon, w.g64, x_o, x_e, WD_ODD, 0, kappa, b_o, 1.0, nullptr, 0, nullptr, st));
  char* rf_e = (char*)w.rf64;
  char* rf_o = rf_e + h64;
  // r_e = kappa H_eo x_o + b_e - x_e ; r_o = kappa H_oe x_e + b_o - x_o
  WD_CK(dsl(c, WD_F64, c.orecon, w.g64, rf_e, x_o, WD_EVEN, 0, kappa, b_e, 1.0, x_e, -1.0,
            &w.sc->res_e, st));
  WD_CK(dsl(c, WD_F64, c.orecon, w.g64, rf_o, x_e, WD_ODD, 0, kappa, b_o, 1.0, x_o, -1.0,
            &w.sc->res_o, st));
  // ---- unpack the solution ----
  double* xdev = x_dev ? x : w.canon_spinor;
  if (!x_dev && !w.canon_spinor) WD_CK(cudaMalloc(&w.canon_spinor, V * 24 * sizeof(double)));
  xdev = x_dev ? x : w.canon_spinor;
  WD_CK(unpack_spinor(xdev, w.x64, g, WD_FULL, WD_F64, st));
  if (P.gauge_fix) WD_CK(rotate_spinor(xdev, xdev, w.gf_omega, g, 1, st));
  if (!x_dev)
    WD_CK(cudaMemcpyAsync(x, xdev, V * 24 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WD_CK(read_scalars(c));
  double rel = bnorm > 0 ? std::sqrt(w.sc_host->res_e + w.sc_host->res_o) / bnorm : 0.0;
  if (status == WD_OK && !(rel <= P.tol)) status = WD_ERR_NOCONV;

  I.iters = iters;
  I.reliable_updates = ru;
  I.status = status;
  I.true_residual = rel;
  I.dslash_calls = c.dslash_calls;
  I.seconds = secs(t0, now());
  I.final_seconds = secs(t_fin, now());
  if (info) *info = I;
  return status;
}

}  // namespace wd
