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

#include <cstdio>
#include <cstring>
#include <map>
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

// Expansion of the transported half spinor t back to four spins, scaled by
// sc and added to acc (sc carries the antiperiodic sign; SC1 marks sc == 1
// known at compile time).
template <int MU, int S, bool SC1, typename R>
__device__ __forceinline__ void expand_add(cx<R> (&acc)[12], const cx<R> (&t)[6], R sc) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    if constexpr (SC1) {
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
    } else {
      const R sp = (R)S * sc;  // S * sc
      acc[c].r = fma(sc, t[c].r, acc[c].r);
      acc[c].i = fma(sc, t[c].i, acc[c].i);
      acc[3 + c].r = fma(sc, t[3 + c].r, acc[3 + c].r);
      acc[3 + c].i = fma(sc, t[3 + c].i, acc[3 + c].i);
      if constexpr (MU == 0) {          // -S i t1 = (S t1.i, -S t1.r)
        acc[6 + c].r = fma(sp, t[3 + c].i, acc[6 + c].r);
        acc[6 + c].i = fma(-sp, t[3 + c].r, acc[6 + c].i);
        acc[9 + c].r = fma(sp, t[c].i, acc[9 + c].r);
        acc[9 + c].i = fma(-sp, t[c].r, acc[9 + c].i);
      } else if constexpr (MU == 1) {   // -S t1, S t0
        acc[6 + c].r = fma(-sp, t[3 + c].r, acc[6 + c].r);
        acc[6 + c].i = fma(-sp, t[3 + c].i, acc[6 + c].i);
        acc[9 + c].r = fma(sp, t[c].r, acc[9 + c].r);
        acc[9 + c].i = fma(sp, t[c].i, acc[9 + c].i);
      } else if constexpr (MU == 2) {   // -S i t0 = (S t0.i, -S t0.r) ; S i t1 = (-S t1.i, S t1.r)
        acc[6 + c].r = fma(sp, t[c].i, acc[6 + c].r);
        acc[6 + c].i = fma(-sp, t[c].r, acc[6 + c].i);
        acc[9 + c].r = fma(-sp, t[3 + c].i, acc[9 + c].r);
        acc[9 + c].i = fma(sp, t[3 + c].r, acc[9 + c].i);
      } else {                          // -S t0, -S t1
        acc[6 + c].r = fma(-sp, t[c].r, acc[6 + c].r);
        acc[6 + c].i = fma(-sp, t[c].i, acc[6 + c].i);
        acc[9 + c].r = fma(-sp, t[3 + c].r, acc[9 + c].r);
        acc[9 + c].i = fma(-sp, t[3 + c].i, acc[9 + c].i);
      }
    }
  }
}

// Half-precision projection on packed (re, im) pairs: the stored values are
// scaled to |v| <= 1, so the rank-2 combination is formed in half2 and only
// the six results are widened; the site scale is applied at accumulation.
template <int MU, int S>
__device__ __forceinline__ void project_h2(const __half2 (&p)[12], __half2 (&h)[6]) {
  // S i p = (-S p.i, S p.r) = swap(p) * (-S, S)
  const __half2 iS = __floats2half2_rn((float)-S, (float)S);
  const __half2 iN = __floats2half2_rn((float)S, (float)-S);  // -S i
#pragma unroll
  for (int c = 0; c < 3; c++) {
    if constexpr (MU == 0) {          // h0 = p0 + S i p3 ; h1 = p1 + S i p2
      h[c] = __hfma2(__lowhigh2highlow(p[9 + c]), iS, p[c]);
      h[3 + c] = __hfma2(__lowhigh2highlow(p[6 + c]), iS, p[3 + c]);
    } else if constexpr (MU == 1) {   // h0 = p0 + S p3 ; h1 = p1 - S p2
      h[c] = S > 0 ? __hadd2(p[c], p[9 + c]) : __hsub2(p[c], p[9 + c]);
      h[3 + c] = S > 0 ? __hsub2(p[3 + c], p[6 + c]) : __hadd2(p[3 + c], p[6 + c]);
    } else if constexpr (MU == 2) {   // h0 = p0 + S i p2 ; h1 = p1 - S i p3
      h[c] = __hfma2(__lowhigh2highlow(p[6 + c]), iS, p[c]);
      h[3 + c] = __hfma2(__lowhigh2highlow(p[9 + c]), iN, p[3 + c]);
    } else {                          // h0 = p0 - S p2 ; h1 = p1 - S p3
      h[c] = S > 0 ? __hsub2(p[c], p[6 + c]) : __hadd2(p[c], p[6 + c]);
      h[3 + c] = S > 0 ? __hsub2(p[3 + c], p[9 + c]) : __hadd2(p[3 + c], p[9 + c]);
    }
  }
}

#ifndef WD_F32X2
#define WD_F32X2 1
#endif
#if WD_F32X2
// t = U h (FWD) or U^+ h for both half-spinor rows at once with packed
// two-wide FP32 FMAs: each link element multiplies row 0 and row 1, so the
// rows are the two lanes (real parts in one pair, imaginary in the other).
template <bool FWD>
__device__ __forceinline__ void su3_mul_f32x2(const cx<float> (&u)[9], const cx<float> (&h)[6],
                                              cx<float> (&t)[6]) {
  float2 hr[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    hr[d] = make_float2(h[d].r, h[3 + d].r);
    hi[d] = make_float2(h[d].i, h[3 + d].i);
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float2 tr = make_float2(0.f, 0.f), ti = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const cx<float> e = FWD ? u[c * 3 + d] : u[d * 3 + c];
      const float2 er = make_float2(e.r, e.r);
      const float2 ei = make_float2(e.i, e.i);
      const float2 en = make_float2(-e.i, -e.i);
      tr = __ffma2_rn(er, hr[d], tr);
      ti = __ffma2_rn(er, hi[d], ti);
      if (FWD) {  // (e.r + i e.i)(h.r + i h.i)
        tr = __ffma2_rn(en, hi[d], tr);
        ti = __ffma2_rn(ei, hr[d], ti);
      } else {    // (e.r - i e.i)(h.r + i h.i)
        tr = __ffma2_rn(ei, hi[d], tr);
        ti = __ffma2_rn(en, hr[d], ti);
      }
    }
    t[c] = mk<float>(tr.x, ti.x);
    t[3 + c] = mk<float>(tr.y, ti.y);
  }
}
#endif

// Load the neighbour spinor and project it into the half spinor h (FP64 and
// FP32 fields; the FP16 hops run their own pipeline, hops_f16).
template <int P, int MU, int S, typename R, bool COH = false>
__device__ __forceinline__ void load_project(cx<R> (&h)[6], const void* __restrict__ in, int nb,
                                             int Vh_pad) {
  static_assert(P != WD_F16, "FP16 hops: hops_f16");
  cx<R> psi[12];
  load_spinor<P, R, COH>(psi, in, nb, Vh_pad);
  project<MU, S>(psi, h);
}

// One hop: neighbour site nb (opposite parity), link in `region` at site lcb.
// FWD: U h ; backward: U^+ h.  flip: the hop crosses the antiperiodic time
// boundary (applied as a sign at accumulation).
// unit: the link is the identity (temporal gauge, time hop off the boundary
// slice): neither loaded nor multiplied.
template <int P, int RC, int MU, int S, bool FWD, typename R, bool COH = false>
__device__ __forceinline__ void hop(cx<R> (&acc)[12], const void* __restrict__ in,
                                    const void* __restrict__ gauge, int nb, int region, int lcb,
                                    bool flip, int Vh_pad, bool unit = false) {
  cx<R> h[6];
  load_project<P, MU, S, R, COH>(h, in, nb, Vh_pad);
  cx<R> t[6];
  if (MU == 3 && unit) {
#pragma unroll
    for (int k = 0; k < 6; k++) t[k] = h[k];
  } else {
    cx<R> u[9];
    load_link<P, RC, R>(u, gauge, region, lcb, Vh_pad);
#if WD_F32X2
    if constexpr (P == WD_F32) {
      su3_mul_f32x2<FWD>(u, h, t);
    } else
#endif
    {
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
    }
  }
  if constexpr (MU == 3) {
    expand_add<MU, S, false>(acc, t, flip ? (R)-1 : (R)1);
  } else {
    expand_add<MU, S, true>(acc, t, (R)1);
  }
}

// ---------------------------------------------------------------------------
// FP16: the hop split into a fetch (raw 128-bit loads into registers) and a
// compute step, so that the kernel keeps the next hops' loads in flight while
// it computes the current one.  FP16 moves half the bytes of FP32 per hop, so
// without this the SM runs out of outstanding loads before HBM saturates.
// ---------------------------------------------------------------------------

struct RawF16 {
  int4 s[3];   // 24 halves of the neighbour spinor (its site scale is loaded apart)
  int4 la;     // link U00 U01 U02 U10
  int2 lb;     // link U11 U12
};

template <bool COH = false>
__device__ __forceinline__ RawF16 fetch_f16(const void* __restrict__ in,
                                            const void* __restrict__ gauge, int nb, int region,
                                            int lcb, int VP, bool unit = false) {
  RawF16 r;
  const int4* p = (const int4*)in;
#pragma unroll
  for (int k = 0; k < 3; k++) r.s[k] = ldin<COH>(p + sbi(nb, k, 3));
  if (!unit) {
    r.la = __ldg((const int4*)gauge + (size_t)region * VP + lcb);
    r.lb = __ldg((const int2*)((const char*)gauge + (size_t)8 * VP * 16) + (size_t)region * VP + lcb);
  } else {
    r.la = make_int4(0, 0, 0, 0);
    r.lb = make_int2(0, 0);
  }
  return r;
}

// Packed half2 complex arithmetic for the FP16 link product.  With
// hx = (-h.i, h.r) = i h:  u h = u.r h + u.i hx, and with hx = (h.i, -h.r) =
// -i h:  conj(u) h = u.r h + u.i hx, so one routine serves U h and U^+ h.
__device__ __forceinline__ __half2 h2_cmac(__half2 u, __half2 h, __half2 hx, __half2 w) {
  w = __hfma2(__low2half2(u), h, w);
  return __hfma2(__high2half2(u), hx, w);
}

// Exact sign and lane moves on a half2 done on the integer pipe (GB300 issues
// packed half FMAs at half the rate of FP32 ones, so the half pipe is kept
// for the arithmetic): h2_sgn flips the sign of the lanes in MASK
// (0x0000ffff: re, 0xffff0000: im); h2_i is i h = (-h.i, h.r), h2_mi is
// -i h = (h.i, -h.r).
__device__ __forceinline__ unsigned h2_bits(__half2 h) {
  unsigned u;
  memcpy(&u, &h, 4);
  return u;
}
__device__ __forceinline__ __half2 h2_from_bits(unsigned u) {
  __half2 h;
  memcpy(&h, &u, 4);
  return h;
}
template <unsigned MASK>
__device__ __forceinline__ __half2 h2_sgn(__half2 h) {
  return h2_from_bits(h2_bits(h) ^ (MASK & 0x80008000u));
}
__device__ __forceinline__ __half2 h2_i(__half2 h) {
  return h2_from_bits(__byte_perm(h2_bits(h), 0, 0x1032) ^ 0x00008000u);
}
__device__ __forceinline__ __half2 h2_mi(__half2 h) {
  return h2_from_bits(__byte_perm(h2_bits(h), 0, 0x1032) ^ 0x80000000u);
}

// conj(a b - c d) on half2 (the SU(3) third row from the first two)
__device__ __forceinline__ __half2 h2_conj_cross(__half2 a, __half2 b, __half2 c, __half2 d) {
  const __half2 bx = h2_i(b);
  const __half2 dx = h2_i(d);
  __half2 x = __hmul2(__low2half2(a), b);
  x = __hfma2(__high2half2(a), bx, x);
  x = __hfma2(__hneg2(__low2half2(c)), d, x);
  x = __hfma2(__hneg2(__high2half2(c)), dx, x);
  return h2_sgn<0xffff0000u>(x);
}

// The transported half spinor t = U h (FWD) or U^+ h in half2 arithmetic:
// the stored spinor is scaled to |v| <= 1 and |U_ij| <= 1, so every partial
// sum stays below 6 in magnitude and each rounding is relative 2^-11, the
// same order as the storage rounding of the FP16 format itself.
template <bool FWD>
__device__ __forceinline__ void transport_h2(const RawF16& r, const __half2 (&h)[6],
                                             __half2 (&t)[6]) {
  __half2 u[9];
  const __half2* ha = reinterpret_cast<const __half2*>(&r.la);
  const __half2* hb = reinterpret_cast<const __half2*>(&r.lb);
#pragma unroll
  for (int j = 0; j < 4; j++) u[j] = ha[j];
  u[4] = hb[0];
  u[5] = hb[1];
  u[6] = h2_conj_cross(u[1], u[5], u[2], u[4]);
  u[7] = h2_conj_cross(u[2], u[3], u[0], u[5]);
  u[8] = h2_conj_cross(u[0], u[4], u[1], u[3]);
  __half2 hx[6];
#pragma unroll
  for (int k = 0; k < 6; k++) hx[k] = FWD ? h2_i(h[k]) : h2_mi(h[k]);
#pragma unroll
  for (int hs = 0; hs < 2; hs++) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      __half2 w = __float2half2_rn(0.f);
#pragma unroll
      for (int d = 0; d < 3; d++) {
        const __half2 e = FWD ? u[c * 3 + d] : u[d * 3 + c];
        w = h2_cmac(e, h[hs * 3 + d], hx[hs * 3 + d], w);
      }
      t[hs * 3 + c] = w;
    }
  }
}

// One FP16 hop: project, transport, expand and accumulate, all in packed
// half2.  rs = (rel, rel), rel = s / smax the neighbour's site scale relative
// to the largest scale of the site's eight neighbours (negated for a hop
// across the antiperiodic time boundary), so every accumulated term is at
// most the size
// of a transported component (below 4) and the eight-hop sums stay below 32:
// no overflow, and a neighbour too small to register in half precision is
// also below the rounding of the result.  The caller applies smax (and the
// kernel's factor a) once, in FP32, after the last hop.
template <int MU, int S, bool FWD>
__device__ __forceinline__ void compute_f16(__half2 (&acc)[12], const RawF16& r, __half2 rs,
                                            bool unit = false) {
  __half2 v[12];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const __half2* q = reinterpret_cast<const __half2*>(&r.s[k]);
#pragma unroll
    for (int j = 0; j < 4; j++) v[4 * k + j] = q[j];
  }
  __half2 hh[6];
  project_h2<MU, S>(v, hh);
  __half2 t[6];
  if (MU == 3 && unit) {
#pragma unroll
    for (int k = 0; k < 6; k++) t[k] = hh[k];
  } else {
    transport_h2<FWD>(r, hh, t);
  }
  // the lower two spins are +-S t or +-S i t of the upper ones (the same
  // expansion as expand_add): with i t = swap(t) * (-1, 1), -S i t = swap(t)
  // * (S, -S)
  const __half2 rn = h2_sgn<0xffffffffu>(rs);
  const __half2 ri = h2_sgn<(S > 0 ? 0xffff0000u : 0x0000ffffu)>(rs);  // (S r, -S r)
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = __hfma2(rs, t[c], acc[c]);
    acc[3 + c] = __hfma2(rs, t[3 + c], acc[3 + c]);
    if constexpr (MU == 0) {          // lower = (-S i t1, -S i t0)
      acc[6 + c] = __hfma2(ri, __lowhigh2highlow(t[3 + c]), acc[6 + c]);
      acc[9 + c] = __hfma2(ri, __lowhigh2highlow(t[c]), acc[9 + c]);
    } else if constexpr (MU == 1) {   // lower = (-S t1, S t0)
      acc[6 + c] = __hfma2(S > 0 ? rn : rs, t[3 + c], acc[6 + c]);
      acc[9 + c] = __hfma2(S > 0 ? rs : rn, t[c], acc[9 + c]);
    } else if constexpr (MU == 2) {   // lower = (-S i t0, S i t1)
      acc[6 + c] = __hfma2(ri, __lowhigh2highlow(t[c]), acc[6 + c]);
      acc[9 + c] = __hfma2(h2_sgn<0xffffffffu>(ri), __lowhigh2highlow(t[3 + c]), acc[9 + c]);
    } else {                          // lower = (-S t0, -S t1)
      acc[6 + c] = __hfma2(S > 0 ? rn : rs, t[c], acc[6 + c]);
      acc[9 + c] = __hfma2(S > 0 ? rn : rs, t[3 + c], acc[9 + c]);
    }
  }
}

// The largest of the eight neighbour scales s (hop order f0 b0 f1 b1 f2 b2
// f3 b3), and the scales relative to it rounded to half, two hops per
// register (rel[k] = (s[2k], s[2k+1]) / smax, the time hops' signs folded
// in).  An all-zero neighbourhood gives smax = 0 and rel = 0.
__device__ __forceinline__ float f16_rel(const float (&s)[8], bool fflip, bool bflip,
                                         __half2 (&rel)[4]) {
  const float m = fmaxf(fmaxf(fmaxf(s[0], s[1]), fmaxf(s[2], s[3])),
                        fmaxf(fmaxf(s[4], s[5]), fmaxf(s[6], s[7])));
  const float inv = m > 0.f ? __frcp_rn(m) : 0.f;
  rel[0] = __floats2half2_rn(s[0] * inv, s[1] * inv);
  rel[1] = __floats2half2_rn(s[2] * inv, s[3] * inv);
  rel[2] = __floats2half2_rn(s[4] * inv, s[5] * inv);
  rel[3] = __floats2half2_rn((fflip ? -s[6] : s[6]) * inv, (bflip ? -s[7] : s[7]) * inv);
  return m;
}

// acc = post * smax * (half2 sums), in FP32
__device__ __forceinline__ void f16_widen(cx<float> (&acc)[12], const __half2 (&ah)[12],
                                          float k) {
#pragma unroll
  for (int j = 0; j < 12; j++) {
    const float2 f = __half22float2(ah[j]);
    acc[j] = mk<float>(k * f.x, k * f.y);
  }
}

// Store k * ah as an FP16 site (the format of store_spinor: values scaled by
// the site's largest |component| m, and m as the site scale) without leaving
// half2 when it can: the largest |component| of ah is found in half2, and
// ah is scaled by 1/max in half2 when that reciprocal is representable
// (max >= 2^-14); a smaller (nonzero) maximum takes the FP32 route.  KEEP:
// kept receives the stored site (for a fused norm).
template <bool KEEP = false>
__device__ __forceinline__ void store_f16_h2(void* base, int cb, int Vh_pad,
                                             const __half2 (&ah)[12], float k,
                                             cx<float> (&kept)[12]) {
  __half2 m2 = __habs2(ah[0]);
#pragma unroll
  for (int j = 1; j < 12; j++) m2 = __hmax2(m2, __habs2(ah[j]));
  const float m = fmaxf(__low2float(m2), __high2float(m2));
  int4* p = (int4*)base;
  float* sc = (float*)((char*)base + (size_t)Vh_pad * 48);
  int4 v[3];
  __half2* h = reinterpret_cast<__half2*>(v);
  if (m >= 6.103515625e-05f) {
    const __half2 inv = __float2half2_rn(k < 0.f ? -__frcp_rn(m) : __frcp_rn(m));
#pragma unroll
    for (int j = 0; j < 12; j++) h[j] = __hmul2(ah[j], inv);
  } else {
    const float inv = m > 0.f ? (k < 0.f ? -1.f : 1.f) / m : 0.f;
#pragma unroll
    for (int j = 0; j < 12; j++) {
      const float2 f = __half22float2(ah[j]);
      h[j] = __floats2half2_rn(f.x * inv, f.y * inv);
    }
  }
#pragma unroll
  for (int j = 0; j < 3; j++) p[sbi(cb, j, 3)] = v[j];
  const float so = m * fabsf(k);
  sc[cb] = so;
  if constexpr (KEEP) {  // what was stored, as load_spinor_rw would read it back
#pragma unroll
    for (int j = 0; j < 12; j++) {
      const float2 f = __half22float2(h[j]);
      kept[j] = mk<float>(f.x * so, f.y * so);
    }
  }
}

#ifndef WD_F16_PREFETCH
#define WD_F16_PREFETCH 2
#endif

// The eight hops of one FP16 site: the eight neighbour scales are loaded
// first, then the loads of the next hops are issued before the current one
// is computed (WD_F16_PREFETCH hops in flight).  The hops are accumulated in
// half2 relative to the largest neighbour scale (compute_f16), which is
// returned: H in at this site = smax * ah.  funit/bunit: the
// forward/backward time link is the identity (temporal gauge).
template <int SF, int SB_, bool COH = false>
__device__ __forceinline__ float hops_f16(__half2 (&ah)[12], const void* __restrict__ in,
                                          const void* __restrict__ ga, int p, int cb, int f0,
                                          int b0, int f1, int b1, int f2, int b2, int f3, int b3,
                                          bool fflip, bool bflip, bool funit, bool bunit, int VP) {
  const int q = 1 - p;
  const float* scl = (const float*)((const char*)in + (size_t)VP * 48);
  float sc[8] = {ldin<COH>(scl + f0), ldin<COH>(scl + b0), ldin<COH>(scl + f1),
                 ldin<COH>(scl + b1), ldin<COH>(scl + f2), ldin<COH>(scl + b2),
                 ldin<COH>(scl + f3), ldin<COH>(scl + b3)};
#pragma unroll
  for (int k = 0; k < 12; k++) ah[k] = __float2half2_rn(0.f);
#define WD_F(nb, reg, lcb) fetch_f16<COH>(in, ga, nb, reg, lcb, VP)
#if WD_F16_PREFETCH >= 3
  RawF16 r0 = WD_F(f0, 0 + p, cb), r1 = WD_F(b0, 0 + q, b0);
  RawF16 r2 = WD_F(f1, 2 + p, cb), r3 = WD_F(b1, 2 + q, b1);
  __half2 rel[4];
  const float smax = f16_rel(sc, fflip, bflip, rel);
  compute_f16<0, SF, true>(ah, r0, __low2half2(rel[0]));
  r0 = WD_F(f2, 4 + p, cb);
  compute_f16<0, SB_, false>(ah, r1, __high2half2(rel[0]));
  r1 = WD_F(b2, 4 + q, b2);
  compute_f16<1, SF, true>(ah, r2, __low2half2(rel[1]));
  r2 = fetch_f16<COH>(in, ga, f3, 6 + p, cb, VP, funit);
  compute_f16<1, SB_, false>(ah, r3, __high2half2(rel[1]));
  r3 = fetch_f16<COH>(in, ga, b3, 6 + q, b3, VP, bunit);
  compute_f16<2, SF, true>(ah, r0, __low2half2(rel[2]));
  compute_f16<2, SB_, false>(ah, r1, __high2half2(rel[2]));
  compute_f16<3, SF, true>(ah, r2, __low2half2(rel[3]), funit);
  compute_f16<3, SB_, false>(ah, r3, __high2half2(rel[3]), bunit);
#elif WD_F16_PREFETCH >= 2
  RawF16 r0 = WD_F(f0, 0 + p, cb), r1 = WD_F(b0, 0 + q, b0);
  RawF16 r2 = WD_F(f1, 2 + p, cb);
  __half2 rel[4];
  const float smax = f16_rel(sc, fflip, bflip, rel);
  compute_f16<0, SF, true>(ah, r0, __low2half2(rel[0]));
  RawF16 r3 = WD_F(b1, 2 + q, b1);
  compute_f16<0, SB_, false>(ah, r1, __high2half2(rel[0]));
  r0 = WD_F(f2, 4 + p, cb);
  compute_f16<1, SF, true>(ah, r2, __low2half2(rel[1]));
  r1 = WD_F(b2, 4 + q, b2);
  compute_f16<1, SB_, false>(ah, r3, __high2half2(rel[1]));
  r2 = fetch_f16<COH>(in, ga, f3, 6 + p, cb, VP, funit);
  compute_f16<2, SF, true>(ah, r0, __low2half2(rel[2]));
  r3 = fetch_f16<COH>(in, ga, b3, 6 + q, b3, VP, bunit);
  compute_f16<2, SB_, false>(ah, r1, __high2half2(rel[2]));
  compute_f16<3, SF, true>(ah, r2, __low2half2(rel[3]), funit);
  compute_f16<3, SB_, false>(ah, r3, __high2half2(rel[3]), bunit);
#else
  RawF16 r0 = WD_F(f0, 0 + p, cb);
  RawF16 r1 = WD_F(b0, 0 + q, b0);
  __half2 rel[4];
  const float smax = f16_rel(sc, fflip, bflip, rel);
  compute_f16<0, SF, true>(ah, r0, __low2half2(rel[0]));
  r0 = WD_F(f1, 2 + p, cb);
  compute_f16<0, SB_, false>(ah, r1, __high2half2(rel[0]));
  r1 = WD_F(b1, 2 + q, b1);
  compute_f16<1, SF, true>(ah, r0, __low2half2(rel[1]));
  r0 = WD_F(f2, 4 + p, cb);
  compute_f16<1, SB_, false>(ah, r1, __high2half2(rel[1]));
  r1 = WD_F(b2, 4 + q, b2);
  compute_f16<2, SF, true>(ah, r0, __low2half2(rel[2]));
  r0 = fetch_f16<COH>(in, ga, f3, 6 + p, cb, VP, funit);
  compute_f16<2, SB_, false>(ah, r1, __high2half2(rel[2]));
  r1 = fetch_f16<COH>(in, ga, b3, 6 + q, b3, VP, bunit);
  compute_f16<3, SF, true>(ah, r0, __low2half2(rel[3]), funit);
  compute_f16<3, SB_, false>(ah, r1, __high2half2(rel[3]), bunit);
#endif
#undef WD_F
  return smax;
}

// TG: links in temporal gauge (compile-time, so that the ordinary kernel keeps
// its register budget)
// BS sites per CTA; the register budget per thread is that of the 128-site
// CTAs for every BS (the same number of resident warps)
template <int P, bool NORM, int BS>
struct DslashMinBlocksBS {
  static constexpr int raw = DslashMinBlocks<P, NORM>::value * DSLASH_BS / BS;
  static constexpr int value = raw < 1 ? 1 : raw;
};

template <int P, int RC, bool DAG, int RED, bool TG, int BS>
__global__ void __launch_bounds__(BS, (DslashMinBlocksBS<P, RED != RED_NONE, BS>::value))
    dslash_kernel(const DslashArgs a) {
  constexpr int NRED = RED == RED_NONE ? 1 : RED == RED_NORM ? 1 : RED == RED_NORM_DOTX ? 3 : 2;
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  pdl_begin();
  const Geom& g = a.g;
  const int cb = blockIdx.x * BS + threadIdx.x;
  R red[NRED];
#pragma unroll
  for (int j = 0; j < NRED; j++) red[j] = (R)0;
  if (cb < g.Vh) {
    const int p = a.parity;
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
    // temporal gauge: U_t(x) = 1 unless x3 = L3-1; the backward link
    // U_t(x - t) is at x3 - 1, the identity unless x3 = 0
    const bool funit = TG && !fflip;
    const bool bunit = TG && !bflip;

    // forward hops use (1 - s gamma), backward (1 + s gamma)
    constexpr int SF = DAG ? -1 : 1;
    constexpr int SB_ = -SF;
    const int q = 1 - p;
    const int VP = g.Vh_pad;

    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = mk<R>(0, 0);

    bool stored = false;
    if constexpr (P == WD_F16) {
      __half2 ah[12];
      const float kf = (float)a.a * hops_f16<SF, SB_>(ah, a.in, a.gauge, p, cb, f0, b0, f1, b1,
                                                      f2, b2, f3, b3, fflip, bflip, funit, bunit,
                                                      VP);
      if (!a.x && !a.y) {
        store_f16_h2<RED != RED_NONE>(a.out, cb, VP, ah, kf, acc);
        stored = true;
      } else {
        f16_widen(acc, ah, kf);
      }
    } else {
      hop<P, RC, 0, SF, true>(acc, a.in, a.gauge, f0, 0 + p, cb, false, VP);
      hop<P, RC, 0, SB_, false>(acc, a.in, a.gauge, b0, 0 + q, b0, false, VP);
      hop<P, RC, 1, SF, true>(acc, a.in, a.gauge, f1, 2 + p, cb, false, VP);
      hop<P, RC, 1, SB_, false>(acc, a.in, a.gauge, b1, 2 + q, b1, false, VP);
      hop<P, RC, 2, SF, true>(acc, a.in, a.gauge, f2, 4 + p, cb, false, VP);
      hop<P, RC, 2, SB_, false>(acc, a.in, a.gauge, b2, 4 + q, b2, false, VP);
      hop<P, RC, 3, SF, true>(acc, a.in, a.gauge, f3, 6 + p, cb, fflip, VP, funit);
      hop<P, RC, 3, SB_, false>(acc, a.in, a.gauge, b3, 6 + q, b3, bflip, VP, bunit);
    }

    if constexpr (P != WD_F16) {  // (the FP16 hops apply a themselves)
      const R ca = (R)a.a;
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = ca * acc[k];
    }
    if (!stored) {
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
      if constexpr (P == WD_F16 && RED != RED_NONE)
        store_spinor_f16<R, true>(a.out, cb, VP, acc);
      else
        store_spinor<P, R>(a.out, cb, VP, acc);
    }
    if constexpr (RED != RED_NONE) {
      // (for FP16, acc now holds what was stored, after rounding to half)
      if constexpr (RED == RED_NORM || RED == RED_NORM_DOTX) red[0] = site_norm2<R>(acc);
      if constexpr (RED == RED_NORM_DOTX) {
        cx<R> v[12];
        load_spinor_rw<P, R>(v, a.x, cb, VP);
        site_cdot(acc, v, red[1], red[2]);
      }
      if constexpr (RED == RED_DOTZ) {
        cx<R> v[12];
        load_spinor_rw<P, R>(v, a.z, cb, VP);
        site_cdot(v, acc, red[0], red[1]);
      }
    }
  }
  // (the launch that follows sums the block partials into norm_out)
  if constexpr (RED != RED_NONE) block_partials<NRED, BS>(red, a.rs.partials);
}

// Launch a hopping kernel (see launch_pdl)
inline cudaError_t launch_hopping(void (*k)(const DslashArgs), dim3 grid, dim3 block,
                                  const DslashArgs& a, cudaStream_t st) {
  return launch_pdl(k, grid, block, st, a);
}

// the non-reducing kernel with BS sites per CTA (64, 128 or 256)
template <int P, int RC, bool DG, bool TG>
cudaError_t launch_dslash_plain_bs(const DslashArgs& a, int bs, cudaStream_t st) {
  const unsigned n = (unsigned)a.g.Vh;
  switch (bs) {
    case 64:
      return launch_hopping(dslash_kernel<P, RC, DG, RED_NONE, TG, 64>, dim3((n + 63) / 64),
                            dim3(64), a, st);
    case 256:
      return launch_hopping(dslash_kernel<P, RC, DG, RED_NONE, TG, 256>, dim3((n + 255) / 256),
                            dim3(256), a, st);
    default:
      return launch_hopping(dslash_kernel<P, RC, DG, RED_NONE, TG, DSLASH_BS>,
                            dim3((n + DSLASH_BS - 1) / DSLASH_BS), dim3(DSLASH_BS), a, st);
  }
}

template <int P, int RC, bool DG, bool TG>
cudaError_t launch_dslash_red_one(const DslashArgs& a, dim3 grid, dim3 block, int bs,
                                  cudaStream_t st) {
  const int mode = a.norm_out ? a.red_mode : RED_NONE;
  switch (mode) {
    case RED_NONE:
      return launch_dslash_plain_bs<P, RC, DG, TG>(a, bs, st);
    case RED_NORM:
      return launch_hopping(dslash_kernel<P, RC, DG, RED_NORM, TG, DSLASH_BS>, grid, block, a, st);
    case RED_NORM_DOTX:
    case RED_DOTZ:
      // the dot-product epilogues serve BiCGstab, which never applies H^+
      if constexpr (!DG) {
        if (mode == RED_NORM_DOTX) {
          if (!a.x) return cudaErrorInvalidValue;
          return launch_hopping(dslash_kernel<P, RC, DG, RED_NORM_DOTX, TG, DSLASH_BS>, grid,
                                block, a, st);
        }
        if (!a.z) return cudaErrorInvalidValue;
        return launch_hopping(dslash_kernel<P, RC, DG, RED_DOTZ, TG, DSLASH_BS>, grid, block, a,
                              st);
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

// a reducing launch is followed by the sum of its block partials
template <int P, int RC, bool DG, bool TG>
cudaError_t launch_dslash_red_tg(const DslashArgs& a, dim3 grid, dim3 block, int bs,
                                 cudaStream_t st) {
  cudaError_t e = launch_dslash_red_one<P, RC, DG, TG>(a, grid, block, bs, st);
  if (e != cudaSuccess || !a.norm_out || a.red_mode == RED_NONE) return e;
  const int nred = a.red_mode == RED_NORM ? 1 : a.red_mode == RED_NORM_DOTX ? 3 : 2;
  return sum_block_partials(nred, a.rs.partials, (int)grid.x, a.norm_out, st);
}

template <int P, int RC, bool DG>
cudaError_t launch_dslash_red(const DslashArgs& a, dim3 grid, dim3 block, int bs,
                              cudaStream_t st) {
  return a.tg ? launch_dslash_red_tg<P, RC, DG, true>(a, grid, block, bs, st)
              : launch_dslash_red_tg<P, RC, DG, false>(a, grid, block, bs, st);
}

template <int P>
cudaError_t launch_dslash_bs(const DslashArgs& a, int recon, bool dagger, int bs,
                             cudaStream_t st) {
  const int BS = DSLASH_BS;
  dim3 grid((a.g.Vh + BS - 1) / BS), block(BS);
  if (recon == 12)
    return dagger ? launch_dslash_red<P, 12, true>(a, grid, block, bs, st)
                  : launch_dslash_red<P, 12, false>(a, grid, block, bs, st);
  if constexpr (P != WD_F16) {
    if (recon == 18)
      return dagger ? launch_dslash_red<P, 18, true>(a, grid, block, bs, st)
                    : launch_dslash_red<P, 18, false>(a, grid, block, bs, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Run-time choice of the CTA size of the non-reducing hopping kernel (64,
// 128 or 256 sites, the same register budget per thread).  A launch shape
// (link format, dagger, temporal gauge, lattice extents) met for the first
// time outside stream capture is timed with each size (CUDA events, one
// warm-up and three launches, on a temporary output, so no caller data is
// written) and the fastest is kept for the life of the process.  Every size
// gives bit-identical fields.  The reducing variants keep 128 sites, so
// that the summation order of their norms does not depend on a timing.
// ---------------------------------------------------------------------------

struct DslashTuneKey {
  int recon, dagger, tg, L[4];
  bool operator<(const DslashTuneKey& o) const {
    const int x[7] = {recon, dagger, tg, L[0], L[1], L[2], L[3]};
    const int y[7] = {o.recon, o.dagger, o.tg, o.L[0], o.L[1], o.L[2], o.L[3]};
    for (int k = 0; k < 7; k++)
      if (x[k] != y[k]) return x[k] < y[k];
    return false;
  }
};

template <int P>
std::map<DslashTuneKey, int>& dslash_tune_table() {
  static std::map<DslashTuneKey, int> t;
  return t;
}

// the tuner's code for the FP16 kernel with the far neighbours staged in
// shared memory (wd_dslash_staged.cu) in place of a CTA size
constexpr int DSLASH_STAGED = 1;

// the staged kernel serves FP16 with 12-real links, no temporal gauge, no
// fused reduction, on lattices whose (z, t) slices hold a multiple of 32
// sites of one parity
template <int P>
bool dslash_staged_ok(const DslashArgs& a, int recon) {
  return P == WD_F16 && recon == 12 && !a.tg && !a.norm_out && (a.g.S2 & 31) == 0;
}

template <int P>
cudaError_t launch_dslash_sel(const DslashArgs& a, int recon, bool dagger, int bs,
                              cudaStream_t st) {
  if (bs == DSLASH_STAGED)
    return launch_dslash_f16_staged(a, recon, dagger, state().wait_limit, st);
  return launch_dslash_bs<P>(a, recon, dagger, bs, st);
}

template <int P>
cudaError_t dslash_block(const DslashArgs& a, int recon, bool dagger, cudaStream_t st, int* bs) {
  *bs = DSLASH_BS;
  if (a.norm_out) return cudaSuccess;
  if (dslash_forced_block()) {
    *bs = dslash_forced_block();
    return cudaSuccess;
  }
  const DslashTuneKey key{recon, dagger ? 1 : 0, a.tg, {a.g.L[0], a.g.L[1], a.g.L[2], a.g.L[3]}};
  auto& tab = dslash_tune_table<P>();
  auto it = tab.find(key);
  if (it != tab.end()) {
    *bs = it->second;
    return cudaSuccess;
  }
  if (a.no_tune || !autotune_enabled()) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return cudaSuccess;
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, spinor_half_bytes(a.g, P)) != cudaSuccess) {
    cudaGetLastError();  // no room to tune: keep the default
    return cudaSuccess;
  }
  DslashArgs t = a;
  t.out = tmp;  // x and y keep pointing at the caller's fields: only read
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // candidates: the three CTA sizes, and for FP16 the staged kernel where
  // the lattice allows it (bit-identical results)
  const int sizes[4] = {64, 128, 256, DSLASH_STAGED};
  const int ncand = dslash_staged_ok<P>(a, recon) ? 4 : 3;
  float us[4] = {0.f, 0.f, 0.f, 0.f};
  int best = DSLASH_BS;
  float best_us = 0.f;
  for (int c = 0; c < ncand && e == cudaSuccess; c++) {
    e = launch_dslash_sel<P>(t, recon, dagger, sizes[c], st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int k = 0; k < 3 && e == cudaSuccess; k++)
      e = launch_dslash_sel<P>(t, recon, dagger, sizes[c], st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    us[c] = ms * 1e3f / 3.f;
    if (best_us == 0.f || us[c] < best_us) {
      best_us = us[c];
      best = sizes[c];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t fe = cudaFree(tmp);
  if (e != cudaSuccess) return e;
  if (fe != cudaSuccess) return fe;
  tab[key] = best;
  char line[256];
  if (ncand == 4)
    std::snprintf(line, sizeof(line),
                  "dslash prec=%d recon=%d dagger=%d tg=%d dims=%dx%dx%dx%d "
                  "us[64,128,256,staged]=%.1f,%.1f,%.1f,%.1f block=%s\n",
                  P, recon, key.dagger, key.tg, key.L[0], key.L[1], key.L[2], key.L[3], us[0],
                  us[1], us[2], us[3],
                  best == DSLASH_STAGED ? "staged"
                  : best == 64          ? "64"
                  : best == 128         ? "128"
                                        : "256");
  else
    std::snprintf(line, sizeof(line),
                  "dslash prec=%d recon=%d dagger=%d tg=%d dims=%dx%dx%dx%d "
                  "us[64,128,256]=%.1f,%.1f,%.1f block=%d\n",
                  P, recon, key.dagger, key.tg, key.L[0], key.L[1], key.L[2], key.L[3], us[0],
                  us[1], us[2], best);
  dslash_tune_record(line);
  *bs = best;
  return cudaSuccess;
}

// Launch one instance; the .cu file of each precision instantiates it.
template <int P>
cudaError_t launch_dslash_prec(const DslashArgs& a, int recon, bool dagger, cudaStream_t st) {
  int bs = DSLASH_BS;
  cudaError_t e = dslash_block<P>(a, recon, dagger, st, &bs);
  if (e != cudaSuccess) return e;
  if (bs == DSLASH_STAGED && !dslash_staged_ok<P>(a, recon)) bs = DSLASH_BS;
  return launch_dslash_sel<P>(a, recon, dagger, bs, st);
}

}  // namespace wd
