// A gauge-covariant nearest-neighbour convolution layer (the learned
// preconditioner; the paper has no such component):
//
//   y(x)[o][a] = sum_{d=0..8} sum_i W_d[o][i] (T_d phi)(x)[i][a]
//
// T_0 phi(x) = phi(x); T_{1+2mu} phi(x) = U_mu(x) phi(x+mu);
// T_{2+2mu} phi(x) = U_mu(x-mu)^+ phi(x-mu), with the antiperiodic time sign
// of the Wilson operator.  W_d acts on the channel index only (a = colour),
// so the layer commutes with gauge transformations.  Complex weights, FP32
// activations, BF16 tensor-core contraction with FP32 accumulation.
//
// Activation layout: the site-blocked layout of the spinor fields with C
// channels x 3 colours per site (complex index c*3 + a, two complexes per
// 16-byte group, NG = 3C/2 groups); a full field is the even half followed by
// the odd half.  With C = 4 this is exactly the packed FP32 spinor.
//
// Per 128-site tile the nine directions are gathered in chunks of K = 16 real
// columns (one direction for 8 input channels, two for 4): each thread
// transports its site's neighbour channels on the CUDA cores and writes them
// as BF16 rows of three shared-memory A tiles (one per colour, K-major, no
// swizzle); one thread then issues three tcgen05.mma (128 x 16 x 16) that
// accumulate into three TMEM accumulators.  Two A buffers alternate, each
// guarded by an mbarrier that the MMA completion arrives on.
#pragma once

#include <cuda_bf16.h>
#include <cstring>

#include "wd_internal.h"
#include "wd_tc.cuh"

namespace wd {

constexpr int NN_TILE = 128;
constexpr int NN_NDIR = 9;
constexpr long NN_SPIN_LIMIT = 1L << 22;

struct NnLayerArgs {
  Geom g;
  const void* gauge;       // packed FP32, 12 reals (the BF16 copy for BF16 activations)
  const char* in;          // CIN channels, full field
  char* out;               // COUT channels, full field
  size_t in_half, out_half;  // bytes per parity half
  const float* w;          // [9][COUT][CIN] complex (re, im)
  int* err;
  // parity restriction (the even-odd preconditioner): only output sites of
  // parity p0 .. p0 + np - 1 are computed; the input of parity zero_in
  // (-1: none) is known to vanish and is never read, so an output site of
  // that parity gets only its self term and one of the other parity only its
  // hops
  int p0 = 0, np = 2, zero_in = -1;
};

__host__ __device__ constexpr size_t nn_half_bytes(const int vh_pad, int C) {
  return ((size_t)vh_pad * C * 24 + 255) / 256 * 256;
}

// the 9 directions: neighbour site (other parity for d > 0), link, sign
struct NnNeighbours {
  int nb[9];
  int lreg[9];
  int lcb[9];
  bool flip[9];
};

__device__ __forceinline__ void nn_neighbours(NnNeighbours& n, int cb, int p, const Geom& g) {
  int x0, x1, x2, x3;
  cb_coords(cb, p, g, x0, x1, x2, x3);
  const int row = cb - (x0 >> 1);
  const int q = 1 - p;
  n.nb[0] = cb;
  n.lreg[0] = -1;
  n.lcb[0] = 0;
  n.flip[0] = false;
  const int f0 = row + ((x0 + 1 == g.L[0] ? 0 : x0 + 1) >> 1);
  const int b0 = row + ((x0 == 0 ? g.L[0] - 1 : x0 - 1) >> 1);
  const int f1 = x1 == g.L[1] - 1 ? cb - (g.L[1] - 1) * g.S1 : cb + g.S1;
  const int b1 = x1 == 0 ? cb + (g.L[1] - 1) * g.S1 : cb - g.S1;
  const int f2 = x2 == g.L[2] - 1 ? cb - (g.L[2] - 1) * g.S2 : cb + g.S2;
  const int b2 = x2 == 0 ? cb + (g.L[2] - 1) * g.S2 : cb - g.S2;
  const int f3 = x3 == g.L[3] - 1 ? cb - (g.L[3] - 1) * g.S3 : cb + g.S3;
  const int b3 = x3 == 0 ? cb + (g.L[3] - 1) * g.S3 : cb - g.S3;
  const int fw[4] = {f0, f1, f2, f3}, bw[4] = {b0, b1, b2, b3};
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    n.nb[1 + 2 * mu] = fw[mu];
    n.lreg[1 + 2 * mu] = 2 * mu + p;
    n.lcb[1 + 2 * mu] = cb;
    n.flip[1 + 2 * mu] = mu == 3 && x3 == g.L[3] - 1;
    n.nb[2 + 2 * mu] = bw[mu];
    n.lreg[2 + 2 * mu] = 2 * mu + q;
    n.lcb[2 + 2 * mu] = bw[mu];
    n.flip[2 + 2 * mu] = mu == 3 && x3 == 0;
  }
}

// load C channels x 3 colours of site cb of a packed activation half
template <int C>
__device__ __forceinline__ void nn_load(cx<float> (&v)[C * 3], const char* half, int cb, int vh_pad) {
  constexpr int NG = 3 * C / 2;
  const float4* p = (const float4*)half;
#pragma unroll
  for (int k = 0; k < NG; k++) {
    float4 q = __ldg(p + sbi(cb, k, NG));
    v[2 * k] = mk<float>(q.x, q.y);
    v[2 * k + 1] = mk<float>(q.z, q.w);
  }
}

template <int C>
__device__ __forceinline__ void nn_store(char* half, int cb, int vh_pad, const cx<float> (&v)[C * 3]) {
  constexpr int NG = 3 * C / 2;
  float4* p = (float4*)half;
#pragma unroll
  for (int k = 0; k < NG; k++)
    p[sbi(cb, k, NG)] = make_float4(v[2 * k].r, v[2 * k].i, v[2 * k + 1].r, v[2 * k + 1].i);
}

// the transported input channels of direction d at this site
template <int C>
__device__ __forceinline__ void nn_transport(cx<float> (&t)[C * 3], const NnLayerArgs& A,
                                             const NnNeighbours& n, int d, int p) {
  const int src_par = d == 0 ? p : 1 - p;
  cx<float> v[C * 3];
  nn_load<C>(v, A.in + src_par * A.in_half, n.nb[d], A.g.Vh_pad);
  if (d == 0) {
#pragma unroll
    for (int k = 0; k < C * 3; k++) t[k] = v[k];
    return;
  }
  cx<float> u[9];
  load_link<WD_F32, 12, float>(u, A.gauge, n.lreg[d], n.lcb[d], A.g.Vh_pad);
  const float s = n.flip[d] ? -1.f : 1.f;
  const bool fwd = (d & 1) != 0;
#pragma unroll
  for (int c = 0; c < C; c++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<float> w = mk<float>(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; b++) {
        if (fwd)
          w = cmadd(u[a * 3 + b], v[c * 3 + b], w);
        else
          w = cjmadd(u[b * 3 + a], v[c * 3 + b], w);
      }
      t[c * 3 + a] = s * w;
    }
  }
}

// Inference layer kernel.  Two threads per site, each transporting four input
// channels of one direction per K = 16 chunk (CIN = 8: channels 4h..4h+3 of
// the chunk's direction; CIN = 4: the whole site for direction 2c + h), so a
// thread holds 12 complex activations instead of 24 and twice as many warps
// hide the gather latency.  The CTA is persistent over 128-site tiles: the
// TMEM accumulators and the BF16 weight tiles are set up once, and a chunk
// counter carried across tiles drives the two A buffers' mbarrier phases.
constexpr int NN_THREADS = 2 * NN_TILE;
#ifndef WD_NN_MINB
#define WD_NN_MINB 3   // CTAs per SM the register budget is sized for
#endif
#ifndef WD_NN_MINB_BF16
#define WD_NN_MINB_BF16 4   // the BF16-activation variants: fewer registers, one more CTA
#endif

// channels c0 .. c0+3 (12 complex, 6 groups) of site cb of a packed half
template <int C>
__device__ __forceinline__ void nn_load4(cx<float> (&v)[12], const char* half, int cb, int c0) {
  constexpr int NG = 3 * C / 2;
  const float4* p = (const float4*)half;
  const int g0 = c0 * 3 / 2;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    float4 q = __ldg(p + sbi(cb, g0 + k, NG));
    v[2 * k] = mk<float>(q.x, q.y);
    v[2 * k + 1] = mk<float>(q.z, q.w);
  }
}

// neighbour checkerboard indices of the nine directions (index 0: the site)
__device__ __forceinline__ void nn_nbr(int (&nb)[NN_NDIR], int& x3, int cb, int p, const Geom& g) {
  int x0, x1, x2;
  cb_coords(cb, p, g, x0, x1, x2, x3);
  const int row = cb - (x0 >> 1);
  nb[0] = cb;
  nb[1] = row + ((x0 + 1 == g.L[0] ? 0 : x0 + 1) >> 1);
  nb[2] = row + ((x0 == 0 ? g.L[0] - 1 : x0 - 1) >> 1);
  nb[3] = x1 == g.L[1] - 1 ? cb - (g.L[1] - 1) * g.S1 : cb + g.S1;
  nb[4] = x1 == 0 ? cb + (g.L[1] - 1) * g.S1 : cb - g.S1;
  nb[5] = x2 == g.L[2] - 1 ? cb - (g.L[2] - 1) * g.S2 : cb + g.S2;
  nb[6] = x2 == 0 ? cb + (g.L[2] - 1) * g.S2 : cb - g.S2;
  nb[7] = x3 == g.L[3] - 1 ? cb - (g.L[3] - 1) * g.S3 : cb + g.S3;
  nb[8] = x3 == 0 ? cb + (g.L[3] - 1) * g.S3 : cb - g.S3;
}

// T_d of four input channels at this site
template <int C>
__device__ __forceinline__ void nn_transport4(cx<float> (&t)[12], const NnLayerArgs& A, int d,
                                              int p, int cb, int n, int x3, int c0) {
  cx<float> v[12];
  nn_load4<C>(v, A.in + (d == 0 ? p : 1 - p) * A.in_half, n, c0);
  if (d == 0) {
#pragma unroll
    for (int k = 0; k < 12; k++) t[k] = v[k];
    return;
  }
  const int mu = (d - 1) >> 1;
  const bool fwd = (d & 1) != 0;
  cx<float> u[9];
  load_link<WD_F32, 12, float>(u, A.gauge, 2 * mu + (fwd ? p : 1 - p), fwd ? cb : n,
                               A.g.Vh_pad);
  const bool flip = mu == 3 && (fwd ? x3 == A.g.L[3] - 1 : x3 == 0);
  const float sg = flip ? -1.f : 1.f;
#pragma unroll
  for (int c = 0; c < 4; c++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<float> w = mk<float>(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; b++) {
        if (fwd)
          w = cmadd(u[a * 3 + b], v[c * 3 + b], w);
        else
          w = cjmadd(u[b * 3 + a], v[c * 3 + b], w);
      }
      t[c * 3 + a] = sg * w;
    }
  }
}

// ---------------------------------------------------------------------------
// BF16 activations (inference inside the solver).  A BF16 activation field
// stores each complex value as one bf16x2 (re, im): C channels x 3 colours
// per site, 12 C bytes, site-blocked in 16-byte groups (NG = 3C/4 groups of
// four complex values; the complex index is c*3 + a as in the FP32 layout).
// BF16 keeps the FP32 exponent range, so the tiny residuals near the end of
// a solve never underflow.
// ---------------------------------------------------------------------------

__host__ __device__ constexpr size_t nn_half_bytes_bf16(const int vh_pad, int C) {
  return ((size_t)vh_pad * C * 12 + 255) / 256 * 256;
}

// channels c0 .. c0+3 (12 complex: three 16-byte groups) of site cb
template <int C>
__device__ __forceinline__ void nn_load4_bf16(__nv_bfloat162 (&v)[12], const char* half, int cb,
                                              int c0) {
  constexpr int NG = 3 * C / 4;
  const int4* p = (const int4*)half;
  const int g0 = c0 * 3 / 4;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int4 q = __ldg(p + sbi(cb, g0 + k, NG));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int j = 0; j < 4; j++) v[4 * k + j] = h[j];
  }
}

// Exact lane moves on a bf16x2 (re low, im high) on the integer pipe:
// bf2_i(v) = i v = (-v.i, v.r); bf2_conj(v) = (v.r, -v.i).
__device__ __forceinline__ __nv_bfloat162 bf2_bits(unsigned x) {
  __nv_bfloat162 h;
  memcpy(&h, &x, 4);
  return h;
}
__device__ __forceinline__ unsigned bf2_u(__nv_bfloat162 h) {
  unsigned x;
  memcpy(&x, &h, 4);
  return x;
}
__device__ __forceinline__ __nv_bfloat162 bf2_i(__nv_bfloat162 v) {
  return bf2_bits(__byte_perm(bf2_u(v), 0, 0x1032) ^ 0x00008000u);
}
__device__ __forceinline__ __nv_bfloat162 bf2_conj(__nv_bfloat162 v) {
  return bf2_bits(bf2_u(v) ^ 0x80000000u);
}

// conj(a b - c d) in bf16x2 arithmetic (the SU(3) third row from the first two)
__device__ __forceinline__ __nv_bfloat162 bf2_conj_cross(__nv_bfloat162 a, __nv_bfloat162 b,
                                                         __nv_bfloat162 c, __nv_bfloat162 d) {
  __nv_bfloat162 x = __hmul2(__low2bfloat162(a), b);
  x = __hfma2(__high2bfloat162(a), bf2_i(b), x);
  x = __hfma2(__hneg2(__low2bfloat162(c)), d, x);
  x = __hfma2(__hneg2(__high2bfloat162(c)), bf2_i(d), x);
  return bf2_conj(x);
}

// The BF16 copy of the 12-real links used by the inference layers: region r
// = 2 mu + parity holds, per site, U00 U01 U02 U10 as four bf16x2 (one int4,
// in the first 8 regions) and U11 U12 as two bf16x2 (one int2, in 8 more
// regions after them): 24 bytes per link, half of the FP32 copy's.
__host__ __device__ constexpr size_t nn_gauge_bytes_bf16(int vh_pad) {
  return (size_t)8 * vh_pad * 24;
}

__device__ __forceinline__ void nn_link_bf16(__nv_bfloat162 (&u)[9], const void* gauge,
                                             int region, int cb, int vh_pad) {
  const int4 la = __ldg((const int4*)gauge + (size_t)region * vh_pad + cb);
  const int2 lb =
      __ldg((const int2*)((const char*)gauge + (size_t)8 * vh_pad * 16) + (size_t)region * vh_pad + cb);
  u[0] = bf2_bits((unsigned)la.x);
  u[1] = bf2_bits((unsigned)la.y);
  u[2] = bf2_bits((unsigned)la.z);
  u[3] = bf2_bits((unsigned)la.w);
  u[4] = bf2_bits((unsigned)lb.x);
  u[5] = bf2_bits((unsigned)lb.y);
  u[6] = bf2_conj_cross(u[1], u[5], u[2], u[4]);
  u[7] = bf2_conj_cross(u[2], u[3], u[0], u[5]);
  u[8] = bf2_conj_cross(u[0], u[4], u[1], u[3]);
}

// T_d of four input channels at this site in packed bf16x2 arithmetic.
// With vx = i v, u v = u.r v + u.i vx and conj(u) v = u.r v - u.i vx, so each
// complex multiply-accumulate is two packed FMAs.  The link comes from the
// BF16 copy (nn_link_bf16), its third row rebuilt in bf16x2.  The input is
// BF16 (BIN) or the packed FP32 field (rounded on load).
template <int C, bool BIN>
__device__ __forceinline__ void nn_transport4_bf16(__nv_bfloat162 (&t)[12], const NnLayerArgs& A,
                                                   int d, int p, int cb, int n, int x3, int c0) {
  __nv_bfloat162 v[12];
  const char* src = A.in + (d == 0 ? p : 1 - p) * A.in_half;
  if constexpr (BIN) {
    nn_load4_bf16<C>(v, src, n, c0);
  } else {
    cx<float> f[12];
    nn_load4<C>(f, src, n, c0);
#pragma unroll
    for (int k = 0; k < 12; k++) v[k] = __floats2bfloat162_rn(f[k].r, f[k].i);
  }
  if (d == 0) {
#pragma unroll
    for (int k = 0; k < 12; k++) t[k] = v[k];
    return;
  }
  const int mu = (d - 1) >> 1;
  const bool fwd = (d & 1) != 0;
  // the link in BF16: rows 0 and 1 loaded, row 2 rebuilt in bf16x2
  __nv_bfloat162 u[9];
  nn_link_bf16(u, A.gauge, 2 * mu + (fwd ? p : 1 - p), fwd ? cb : n, A.g.Vh_pad);
  // the antiperiodic sign of a hop across the time boundary, applied to the
  // result as a sign-bit flip (exact, as a negated link would be)
  const bool flip = mu == 3 && (fwd ? x3 == A.g.L[3] - 1 : x3 == 0);
  const unsigned sgn = flip ? 0x80008000u : 0u;
  // ur[k] = (u.r, u.r), ui[k] = (u.i, u.i) of the element the product needs
  __nv_bfloat162 ur[9], ui[9];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const __nv_bfloat162 e = fwd ? u[a * 3 + b] : u[b * 3 + a];
      ur[a * 3 + b] = __low2bfloat162(e);
      ui[a * 3 + b] = __high2bfloat162(e);
    }
  const __nv_bfloat162 zero = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < 4; c++) {
    // vx = i v (U v) or -i v (U^+ v): a lane swap and a sign-bit flip on the
    // integer pipe (the packed BF16 FMAs issue at half the FP32 rate)
    __nv_bfloat162 vx[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
      unsigned x;
      memcpy(&x, &v[c * 3 + b], 4);
      x = __byte_perm(x, 0, 0x1032) ^ (fwd ? 0x00008000u : 0x80000000u);
      memcpy(&vx[b], &x, 4);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      __nv_bfloat162 w = zero;
#pragma unroll
      for (int b = 0; b < 3; b++) {
        w = __hfma2(ur[a * 3 + b], v[c * 3 + b], w);
        w = __hfma2(ui[a * 3 + b], vx[b], w);
      }
      unsigned y;
      memcpy(&y, &w, 4);
      y ^= sgn;
      memcpy(&t[c * 3 + a], &y, 4);
    }
  }
}

template <int CIN, int COUT, bool BIN = false, bool BOUT = false>
__global__ void __launch_bounds__(NN_THREADS, (BIN || BOUT) ? WD_NN_MINB_BF16 : WD_NN_MINB)
    nn_layer_kernel(const NnLayerArgs A, int ntiles) {
  static_assert(CIN == 4 || CIN == 8, "4 or 8 input channels");
  static_assert(COUT == 4 || COUT == 8, "4 or 8 output channels");
  constexpr int DPC = 16 / (2 * CIN);                  // directions per K = 16 chunk
  constexpr int NCHUNK = (NN_NDIR + DPC - 1) / DPC;
  constexpr int NPAD = 16;                             // N of the MMA (2 COUT <= 16)
  constexpr uint32_t ABUF = NN_TILE * 16 * 2;          // one colour's A chunk, bytes
  __shared__ __align__(128) unsigned char sA[2][3][ABUF];
  __shared__ __align__(128) unsigned char sB[NCHUNK][NPAD * 16 * 2];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int s = tid & (NN_TILE - 1);   // site of the tile = A row = TMEM lane
  const int hh = tid >> 7;             // which half of the chunk's K columns
  const Geom& g = A.g;
  const int tpp = (g.Vh + NN_TILE - 1) / NN_TILE;  // tiles per parity

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 64);
    tmem_relinquish();
  }
  // weights -> BF16 B^T chunks (real form of the complex product), once per CTA
  for (int e = tid; e < NCHUNK * NPAD * 16; e += NN_THREADS) {
    const int c = e / (NPAD * 16), rem = e - c * NPAD * 16;
    const int n = rem / 16, k = rem - n * 16;
    const int j = k / (2 * CIN), i = (k / 2) % CIN, ri = k & 1;
    const int o = n >> 1, ro = n & 1;
    const int d = c * DPC + j;
    float val = 0.f;
    if (d < NN_NDIR && o < COUT) {
      const float wr = A.w[((d * COUT + o) * CIN + i) * 2];
      const float wi = A.w[((d * COUT + o) * CIN + i) * 2 + 1];
      // Y.re = Xr Wr - Xi Wi ; Y.im = Xr Wi + Xi Wr
      val = ro == 0 ? (ri == 0 ? wr : -wi) : (ri == 0 ? wi : wr);
    }
    *(__nv_bfloat16*)(sB[c] + kmajor_offset(n, k, 16)) = __float2bfloat16_rn(val);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = make_idesc_bf16(NN_TILE, NPAD);
  const int c0 = CIN == 8 ? 4 * hh : 0;
  bool ok = true;
  uint32_t G = 0;  // chunks issued by this CTA so far

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int pt = tile / tpp;
    const int p = A.p0 + pt;
    const int cb = (tile - pt * tpp) * NN_TILE + s;
    const bool valid = cb < g.Vh;
    const bool skip_self = A.zero_in == p, skip_hops = A.zero_in == 1 - p;
    int nb[NN_NDIR];
    int x3 = 0;
    if (valid) nn_nbr(nb, x3, cb, p, g);
    // a tile whose hops vanish (its input parity is zero) needs the chunk of
    // the self term only (chunk 0); the condition is the same in the whole CTA
    const int nch = skip_hops ? 1 : NCHUNK;
#pragma unroll
    for (int c = 0; c < NCHUNK; c++) {
      if (c >= nch) break;
      const uint32_t buf = G & 1u;
      if (G >= 2) ok = mbar_wait_bounded(&bar[buf], ((G - 2) >> 1) & 1u, NN_SPIN_LIMIT) && ok;
      const int d = CIN == 8 ? c : 2 * c + hh;
      // the neighbour index by compile-time subscripts only (nb stays in registers)
      int n;
      if constexpr (CIN == 8) {
        n = nb[c];
      } else {
        n = hh ? nb[2 * c + 1 < NN_NDIR ? 2 * c + 1 : 0] : nb[2 * c];
      }
      const bool live = valid && d < NN_NDIR && !(d == 0 ? skip_self : skip_hops);
      if constexpr (BIN || BOUT) {
        // BF16 inference path: transport in packed bf16x2, stored as is
        __nv_bfloat162 t[12];
        if (live) {
          nn_transport4_bf16<CIN, BIN>(t, A, d, p, cb, n, x3, c0);
        } else {
#pragma unroll
          for (int k = 0; k < 12; k++) t[k] = __floats2bfloat162_rn(0.f, 0.f);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int k = 2 * (4 * hh + i);
            *(__nv_bfloat162*)(sA[buf][a] + kmajor_offset(s, k, 16)) = t[i * 3 + a];
          }
        }
      } else {
        cx<float> t[12];
        if (live) {
          nn_transport4<CIN>(t, A, d, p, cb, n, x3, c0);
        } else {
#pragma unroll
          for (int k = 0; k < 12; k++) t[k] = mk<float>(0.f, 0.f);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int k = 2 * (4 * hh + i);
            __nv_bfloat162 h = __floats2bfloat162_rn(t[i * 3 + a].r, t[i * 3 + a].i);
            *(__nv_bfloat162*)(sA[buf][a] + kmajor_offset(s, k, 16)) = h;
          }
        }
      }
      fence_smem_to_async();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint64_t bd = make_smem_desc(smem_u32(sB[c]), 128, 256);
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const uint64_t ad = make_smem_desc(smem_u32(sA[buf][a]), 128, 256);
          tc_mma_bf16(tbase + (uint32_t)(a * NPAD), ad, bd, idesc, c > 0 ? 1u : 0u);
        }
        tc_commit(&bar[buf]);
      }
      G++;
    }
    // the tile's last commit covers every MMA issued before it
    ok = mbar_wait_bounded(&bar[(G - 1) & 1u], ((G - 1) >> 1) & 1u, NN_SPIN_LIMIT) && ok;
    // tcgen05.ld is warp-collective: decide once for the whole CTA
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (!ok) break;
    if (warp < 4) {
      cx<float> y[COUT * 3];
#pragma unroll
      for (int a = 0; a < 3; a++) {
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a * NPAD), v);
#pragma unroll
        for (int o = 0; o < COUT; o++) y[o * 3 + a] = mk<float>(v[2 * o], v[2 * o + 1]);
      }
      if (valid) {
        if constexpr (BOUT) {
          // COUT x 3 complex values as bf16x2, four per 16-byte group
          constexpr int NG = 3 * COUT / 4;
          int4* q = (int4*)(A.out + p * A.out_half);
#pragma unroll
          for (int k = 0; k < NG; k++) {
            __nv_bfloat162 h[4];
#pragma unroll
            for (int j = 0; j < 4; j++) h[j] = __floats2bfloat162_rn(y[4 * k + j].r, y[4 * k + j].i);
            q[sbi(cb, k, NG)] = *reinterpret_cast<const int4*>(h);
          }
        } else {
          nn_store<COUT>(A.out + p * A.out_half, cb, g.Vh_pad, y);
        }
      }
    }
    // the next tile's first MMA is issued after a __syncthreads that follows
    // these TMEM reads
    tc_fence_before();
  }
  if (!ok) {
    if (tid == 0) atomicExch(A.err, 1);
    // give MMAs still in flight a second bounded wait before TMEM is freed
    if (G > 0) mbar_wait_bounded(&bar[(G - 1) & 1u], ((G - 1) >> 1) & 1u, NN_SPIN_LIMIT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 64);
}

// ---------------------------------------------------------------------------
// Inference kernel with one thread per site (BF16 activations, the flexible
// CG's preconditioner).  Each thread transports all input channels of its
// site for a chunk's directions, so the link of a (site, direction) is
// loaded, rebuilt and broadcast once (the two-thread kernel above does it in
// both threads), and each per-chunk CTA barrier joins 4 warps instead of 8.
// Same chunks, A layout, MMAs, TMEM accumulators and epilogue as above, and
// bit-identical results.  Measured against the two-thread kernel on the
// learned-preconditioner solve (32^3x64): 0.206 -> 0.200 s at 80 registers
// (6 CTAs per SM); 72 and 64 registers spill and are slower, and loading a
// chunk ahead (30 more registers) spills or costs residency: 0.203-0.251 s.
// ---------------------------------------------------------------------------

#ifndef WD_NN_MINB_INF
#define WD_NN_MINB_INF 6   // 128-thread CTAs per SM the register budget is sized for
#endif

// the link of direction d > 0 at this site, as the broadcasts the product
// needs (ur = (u.r, u.r), ui = (u.i, u.i) of U (forward) or U^+ (backward)),
// and the sign-bit mask of the antiperiodic boundary
struct NnLinkBf {
  __nv_bfloat162 ur[9], ui[9];
  unsigned sgn;
  bool fwd;
};

__device__ __forceinline__ void nn_link_prep_bf16(NnLinkBf& L, const NnLayerArgs& A, int d, int p,
                                                  int cb, int n, int x3) {
  const int mu = (d - 1) >> 1;
  L.fwd = (d & 1) != 0;
  __nv_bfloat162 u[9];
  nn_link_bf16(u, A.gauge, 2 * mu + (L.fwd ? p : 1 - p), L.fwd ? cb : n, A.g.Vh_pad);
  const bool flip = mu == 3 && (L.fwd ? x3 == A.g.L[3] - 1 : x3 == 0);
  L.sgn = flip ? 0x80008000u : 0u;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const __nv_bfloat162 e = L.fwd ? u[a * 3 + b] : u[b * 3 + a];
      L.ur[a * 3 + b] = __low2bfloat162(e);
      L.ui[a * 3 + b] = __high2bfloat162(e);
    }
}

// four channels (c0 .. c0+3) of the neighbour n of direction d (0: the site
// itself), transported with L, written as the A-row columns 8 h .. 8 h + 7
// of row s (one bf16x2 per complex value, per colour tile)
template <int C, bool BIN>
__device__ __forceinline__ void nn_hop4_rows(unsigned char (&sAb)[3][NN_TILE * 16 * 2],
                                             const NnLayerArgs& A, const NnLinkBf& L, int d,
                                             int p, int n, int c0, int h, int s, bool live) {
  __nv_bfloat162 t[12];
  if (!live) {
#pragma unroll
    for (int k = 0; k < 12; k++) t[k] = __floats2bfloat162_rn(0.f, 0.f);
  } else {
    __nv_bfloat162 v[12];
    const char* src = A.in + (d == 0 ? p : 1 - p) * A.in_half;
    if constexpr (BIN) {
      nn_load4_bf16<C>(v, src, n, c0);
    } else {
      cx<float> f[12];
      nn_load4<C>(f, src, n, c0);
#pragma unroll
      for (int k = 0; k < 12; k++) v[k] = __floats2bfloat162_rn(f[k].r, f[k].i);
    }
    if (d == 0) {
#pragma unroll
      for (int k = 0; k < 12; k++) t[k] = v[k];
    } else {
      const __nv_bfloat162 zero = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        __nv_bfloat162 vx[3];
#pragma unroll
        for (int b = 0; b < 3; b++)
          vx[b] = bf2_bits(__byte_perm(bf2_u(v[c * 3 + b]), 0, 0x1032) ^
                           (L.fwd ? 0x00008000u : 0x80000000u));
#pragma unroll
        for (int a = 0; a < 3; a++) {
          __nv_bfloat162 w = zero;
#pragma unroll
          for (int b = 0; b < 3; b++) {
            w = __hfma2(L.ur[a * 3 + b], v[c * 3 + b], w);
            w = __hfma2(L.ui[a * 3 + b], vx[b], w);
          }
          t[c * 3 + a] = bf2_bits(bf2_u(w) ^ L.sgn);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int i = 0; i < 4; i++)
      *(__nv_bfloat162*)(sAb[a] + kmajor_offset(s, 2 * (4 * h + i), 16)) = t[i * 3 + a];
}

template <int CIN, int COUT, bool BIN, bool BOUT>
__global__ void __launch_bounds__(NN_TILE, WD_NN_MINB_INF)
    nn_infer_kernel(const NnLayerArgs A, int ntiles) {
  static_assert(CIN == 4 || CIN == 8, "4 or 8 input channels");
  static_assert(COUT == 4 || COUT == 8, "4 or 8 output channels");
  constexpr int DPC = 16 / (2 * CIN);                  // directions per K = 16 chunk
  constexpr int NCHUNK = (NN_NDIR + DPC - 1) / DPC;
  constexpr int NPAD = 16;                             // N of the MMA (2 COUT <= 16)
  constexpr uint32_t ABUF = NN_TILE * 16 * 2;          // one colour's A chunk, bytes
  __shared__ __align__(128) unsigned char sA[2][3][ABUF];
  __shared__ __align__(128) unsigned char sB[NCHUNK][NPAD * 16 * 2];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int s = tid;  // site of the tile = A row = TMEM lane
  const Geom& g = A.g;
  const int tpp = (g.Vh + NN_TILE - 1) / NN_TILE;  // tiles per parity

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 64);
    tmem_relinquish();
  }
  // weights -> BF16 B^T chunks (real form of the complex product), once per CTA
  for (int e = tid; e < NCHUNK * NPAD * 16; e += NN_TILE) {
    const int c = e / (NPAD * 16), rem = e - c * NPAD * 16;
    const int nn = rem / 16, k = rem - nn * 16;
    const int j = k / (2 * CIN), i = (k / 2) % CIN, ri = k & 1;
    const int o = nn >> 1, ro = nn & 1;
    const int d = c * DPC + j;
    float val = 0.f;
    if (d < NN_NDIR && o < COUT) {
      const float wr = A.w[((d * COUT + o) * CIN + i) * 2];
      const float wi = A.w[((d * COUT + o) * CIN + i) * 2 + 1];
      // Y.re = Xr Wr - Xi Wi ; Y.im = Xr Wi + Xi Wr
      val = ro == 0 ? (ri == 0 ? wr : -wi) : (ri == 0 ? wi : wr);
    }
    *(__nv_bfloat16*)(sB[c] + kmajor_offset(nn, k, 16)) = __float2bfloat16_rn(val);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = make_idesc_bf16(NN_TILE, NPAD);
  bool ok = true;
  uint32_t G = 0;  // chunks issued by this CTA so far

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int pt = tile / tpp;
    const int p = A.p0 + pt;
    const int cb = (tile - pt * tpp) * NN_TILE + s;
    const bool valid = cb < g.Vh;
    const bool skip_self = A.zero_in == p, skip_hops = A.zero_in == 1 - p;
    int nb[NN_NDIR];
    int x3 = 0;
    if (valid) nn_nbr(nb, x3, cb, p, g);
    // a tile whose hops vanish needs the self-term chunk only (the condition
    // is the same in the whole CTA)
    const int nch = skip_hops ? 1 : NCHUNK;
#pragma unroll
    for (int c = 0; c < NCHUNK; c++) {
      if (c >= nch) break;
      const uint32_t buf = G & 1u;
      if (G >= 2) ok = mbar_wait_bounded(&bar[buf], ((G - 2) >> 1) & 1u, NN_SPIN_LIMIT) && ok;
      NnLinkBf L;
      if constexpr (CIN == 8) {
        // one direction, its link prepared once for both channel halves
        const int d = c;
        const bool live = valid && !(d == 0 ? skip_self : skip_hops);
        if (live && d > 0) nn_link_prep_bf16(L, A, d, p, cb, nb[c], x3);
        nn_hop4_rows<CIN, BIN>(sA[buf], A, L, d, p, nb[c], 0, 0, s, live);
        nn_hop4_rows<CIN, BIN>(sA[buf], A, L, d, p, nb[c], 4, 1, s, live);
      } else {
        // two directions of all four channels
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int d = 2 * c + h;
          if (d < NN_NDIR) {
            const bool live = valid && !(d == 0 ? skip_self : skip_hops);
            if (live && d > 0) nn_link_prep_bf16(L, A, d, p, cb, nb[d], x3);
            nn_hop4_rows<CIN, BIN>(sA[buf], A, L, d, p, nb[d], 0, h, s, live);
          } else {
            nn_hop4_rows<CIN, BIN>(sA[buf], A, L, 0, p, cb, 0, h, s, false);
          }
        }
      }
      fence_smem_to_async();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint64_t bd = make_smem_desc(smem_u32(sB[c]), 128, 256);
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const uint64_t ad = make_smem_desc(smem_u32(sA[buf][a]), 128, 256);
          tc_mma_bf16(tbase + (uint32_t)(a * NPAD), ad, bd, idesc, c > 0 ? 1u : 0u);
        }
        tc_commit(&bar[buf]);
      }
      G++;
    }
    // the tile's last commit covers every MMA issued before it
    ok = mbar_wait_bounded(&bar[(G - 1) & 1u], ((G - 1) >> 1) & 1u, NN_SPIN_LIMIT) && ok;
    // tcgen05.ld is warp-collective: decide once for the whole CTA
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (!ok) break;
    cx<float> y[COUT * 3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a * NPAD), v);
#pragma unroll
      for (int o = 0; o < COUT; o++) y[o * 3 + a] = mk<float>(v[2 * o], v[2 * o + 1]);
    }
    if (valid) {
      if constexpr (BOUT) {
        constexpr int NG = 3 * COUT / 4;
        int4* q = (int4*)(A.out + p * A.out_half);
#pragma unroll
        for (int k = 0; k < NG; k++) {
          __nv_bfloat162 hv[4];
#pragma unroll
          for (int j = 0; j < 4; j++)
            hv[j] = __floats2bfloat162_rn(y[4 * k + j].r, y[4 * k + j].i);
          q[sbi(cb, k, NG)] = *reinterpret_cast<const int4*>(hv);
        }
      } else {
        nn_store<COUT>(A.out + p * A.out_half, cb, g.Vh_pad, y);
      }
    }
    // the next tile's first MMA is issued after a __syncthreads that follows
    // these TMEM reads
    tc_fence_before();
  }
  if (!ok) {
    if (tid == 0) atomicExch(A.err, 1);
    // give MMAs still in flight a second bounded wait before TMEM is freed
    if (G > 0) mbar_wait_bounded(&bar[(G - 1) & 1u], ((G - 1) >> 1) & 1u, NN_SPIN_LIMIT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 64);
}

}  // namespace wd
