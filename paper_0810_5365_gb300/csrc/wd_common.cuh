// Device-side building blocks shared by the libwd kernels: lattice geometry,
// the site-blocked packed field formats, complex arithmetic and the
// deterministic FP64 block reduction.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include <type_traits>

#include "../../include/wd.h"

namespace wd {

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------

// Sites per block of the site-blocked structure-of-arrays layout.  A block of
// 32 consecutive checkerboard sites stores component group k of all its sites
// contiguously, so one warp reading one group issues a single 512-byte (FP32)
// or 1024-byte (FP64) fully coalesced request of 128-bit vectors.
constexpr int SB = 32;

// Exact division by an invariant d for 0 <= n < 2^31 by one 64-bit multiply
// and a shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with s = ceil(log2 d) and M = ceil(2^(32+s)/d),
// floor(n/d) = (n * M) >> (32 + s), since the rounding error of M contributes
// less than n / 2^(32+s) < 1/(2d).
struct FastDiv {
  unsigned long long M;
  int shift;  // 32 + s
  int d;
};

inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  int s = 0;
  while ((1LL << s) < d) s++;
  unsigned __int128 num = (unsigned __int128)1 << (32 + s);
  f.M = (unsigned long long)((num + (unsigned)d - 1) / (unsigned)d);
  f.shift = 32 + s;
  f.d = d;
  return f;
}

__host__ __device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return (int)(((unsigned long long)(unsigned)n * f.M) >> f.shift);
}

struct Geom {
  int L[4];    // extents
  int Lh0;     // L0 / 2
  int Vh;      // sites per parity
  int Vh_pad;  // Vh rounded up to a multiple of SB
  int S1;      // checkerboard stride of +y  (Lh0)
  int S2;      // checkerboard stride of +z  (Lh0 * L1)
  int S3;      // checkerboard stride of +t  (Lh0 * L1 * L2)
  FastDiv dLh0, dL1, dL2;
};

inline Geom make_geom(const int d[4]) {
  Geom g;
  for (int i = 0; i < 4; i++) g.L[i] = d[i];
  g.Lh0 = d[0] / 2;
  long long V = (long long)d[0] * d[1] * d[2] * d[3];
  g.Vh = (int)(V / 2);
  g.Vh_pad = (g.Vh + SB - 1) / SB * SB;
  g.S1 = g.Lh0;
  g.S2 = g.Lh0 * d[1];
  g.S3 = g.Lh0 * d[1] * d[2];
  g.dLh0 = make_fastdiv(g.Lh0);
  g.dL1 = make_fastdiv(d[1]);
  g.dL2 = make_fastdiv(d[2]);
  return g;
}

// Checkerboard site cb of parity p -> coordinates (x0..x3).
__host__ __device__ __forceinline__ void cb_coords(int cb, int p, const Geom& g, int& x0, int& x1, int& x2,
                                          int& x3) {
  const int r0 = fdiv(cb, g.dLh0);
  const int xh = cb - r0 * g.Lh0;
  const int r1 = fdiv(r0, g.dL1);
  x1 = r0 - r1 * g.L[1];
  x3 = fdiv(r1, g.dL2);
  x2 = r1 - x3 * g.L[2];
  x0 = 2 * xh + ((p + x1 + x2 + x3) & 1);
}

// vector index of component group k (of NC) of checkerboard site cb
__host__ __device__ __forceinline__ size_t sbi(int cb, int k, int NC) {
  return ((size_t)(cb >> 5) * NC + k) * SB + (cb & (SB - 1));
}

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------

template <typename R>
struct cx {
  R r, i;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R r, R i) { cx<R> c; c.r = r; c.i = i; return c; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.r + b.r, a.i + b.i); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.r - b.r, a.i - b.i); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.r, s * a.i); }
// i * a
template <typename R>
__device__ __forceinline__ cx<R> ti(cx<R> a) { return mk(-a.i, a.r); }
// a * b
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
// acc + a * b
template <typename R>
__device__ __forceinline__ cx<R> cmadd(cx<R> a, cx<R> b, cx<R> acc) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(-a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i);
  acc.i = fma(a.i, b.r, acc.i);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cjmadd(cx<R> a, cx<R> b, cx<R> acc) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i);
  acc.i = fma(-a.i, b.r, acc.i);
  return acc;
}
// conj(a * b - c * d)
template <typename R>
__device__ __forceinline__ cx<R> conj_cross(cx<R> a, cx<R> b, cx<R> c, cx<R> d) {
  R re = a.r * b.r - a.i * b.i - (c.r * d.r - c.i * d.i);
  R im = a.r * b.i + a.i * b.r - (c.r * d.i + c.i * d.r);
  return mk(re, -im);
}

// ---------------------------------------------------------------------------
// per-site reductions: the 24 terms of one site are summed in the working
// precision R.  The kernels that fuse a reduction keep summing in R over the
// sites of a warp or block, and the per-block (or per-warp) partials are
// summed in FP64.  GB300 issues FP64 at 1/64 of its FP32 rate: a sum over
// sites in FP64 (a shuffle tree of DADDs per warp) costs more than the
// memory traffic of the kernels that fuse these reductions.
// ---------------------------------------------------------------------------

// the arithmetic type of a storage precision (FP32 for FP16 storage)
template <int P>
using real_of = typename std::conditional<P == WD_F64, double, float>::type;

template <typename T = double, typename R>
__device__ __forceinline__ T site_norm2(const cx<R> (&v)[12]) {
  R t = (R)0;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    t = fma(v[k].r, v[k].r, t);
    t = fma(v[k].i, v[k].i, t);
  }
  return (T)t;
}

// re + i im += sum_k conj(a_k) b_k
template <typename R, typename T>
__device__ __forceinline__ void site_cdot(const cx<R> (&a)[12], const cx<R> (&b)[12], T& re,
                                          T& im) {
  R r = (R)0, i = (R)0;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    r = fma(a[k].r, b[k].r, r);
    r = fma(a[k].i, b[k].i, r);
    i = fma(a[k].r, b[k].i, i);
    i = fma(-a[k].i, b[k].r, i);
  }
  re += (T)r;
  im += (T)i;
}

// ---------------------------------------------------------------------------
// packed spinor formats (per parity; Vh_pad sites)
//   WD_F64: NC = 12 double2, group k = complex component k = spin*3 + colour
//   WD_F32: NC =  6 float4,  group k = components 2k, 2k+1
//   WD_F16: NC =  3 int4,    group k = components 4k..4k+3 as half2 (re, im),
//           followed by float scale[Vh_pad]; value = half * scale
// ---------------------------------------------------------------------------

template <int P> struct SpinorFmt;
template <> struct SpinorFmt<WD_F64> { static constexpr size_t bytes_per_site = 192; };
template <> struct SpinorFmt<WD_F32> { static constexpr size_t bytes_per_site = 96; };
template <> struct SpinorFmt<WD_F16> { static constexpr size_t bytes_per_site = 52; };

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline size_t spinor_half_bytes(const Geom& g, int prec) {
  size_t per = prec == WD_F64 ? 192 : prec == WD_F32 ? 96 : 52;
  return round_up((size_t)g.Vh_pad * per, 256);
}

// Programmatic dependent launch.  launch_dependents lets the next kernel of
// the stream be scheduled once every CTA of this grid has started (its CTAs
// then fill the SM slots that this grid's last wave frees); wait blocks until
// the previous kernel of the stream has completed and its writes are
// visible.  A kernel calls this before its first global memory access, so it
// never reads or writes anything its predecessor may still touch.  Both are
// no-ops for a launch without the programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;\n\tgriddepcontrol.wait;\n" ::: "memory");
}

// A load of an input field.  COH = false: the read-only data path (the field
// is not written while the kernel runs).  COH = true: an ordinary coherent
// load, for a kernel that reads fields written earlier in the same launch by
// other CTAs (after a grid barrier).
template <bool COH, typename T>
__device__ __forceinline__ T ldin(const T* p) {
  if constexpr (COH)
    return __ldca(p);
  else
    return __ldg(p);
}

// Load the 12 complex components of site cb as type R.
template <int P, typename R, bool COH = false>
__device__ __forceinline__ void load_spinor(cx<R> (&s)[12], const void* base, int cb, int Vh_pad) {
  if constexpr (P == WD_F64) {
    const double2* p = (const double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = ldin<COH>(p + sbi(cb, k, 12));
      s[k] = mk<R>((R)v.x, (R)v.y);
    }
  } else if constexpr (P == WD_F32) {
    const float4* p = (const float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = ldin<COH>(p + sbi(cb, k, 6));
      s[2 * k] = mk<R>((R)v.x, (R)v.y);
      s[2 * k + 1] = mk<R>((R)v.z, (R)v.w);
    }
  } else {
    const int4* p = (const int4*)base;
    const float* sc = (const float*)((const char*)base + (size_t)Vh_pad * 48);
    float scale = ldin<COH>(sc + cb);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      int4 v = ldin<COH>(p + sbi(cb, k, 3));
      const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        float2 f = __half22float2(h[j]);
        s[4 * k + j] = mk<R>((R)(f.x * scale), (R)(f.y * scale));
      }
    }
  }
}

// Plain (cached) load variant for fields that this kernel also writes
// (x, y operands that may alias out): no read-only path.
template <int P, typename R>
__device__ __forceinline__ void load_spinor_rw(cx<R> (&s)[12], const void* base, int cb, int Vh_pad) {
  if constexpr (P == WD_F64) {
    const double2* p = (const double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = p[sbi(cb, k, 12)];
      s[k] = mk<R>((R)v.x, (R)v.y);
    }
  } else if constexpr (P == WD_F32) {
    const float4* p = (const float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = p[sbi(cb, k, 6)];
      s[2 * k] = mk<R>((R)v.x, (R)v.y);
      s[2 * k + 1] = mk<R>((R)v.z, (R)v.w);
    }
  } else {
    const int4* p = (const int4*)base;
    const float* sc = (const float*)((const char*)base + (size_t)Vh_pad * 48);
    float scale = sc[cb];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      int4 v = p[sbi(cb, k, 3)];
      const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        float2 f = __half22float2(h[j]);
        s[4 * k + j] = mk<R>((R)(f.x * scale), (R)(f.y * scale));
      }
    }
  }
}

// An FP16 site: the values scaled by the site's largest |real component| m,
// rounded to half, and m as the site scale.  KEEP: s is overwritten with
// what was stored (the rounded values times m, as load_spinor_rw would read
// them back), for a norm or dot product of the stored field.
template <typename R, bool KEEP>
__device__ __forceinline__ void store_spinor_f16(void* base, int cb, int Vh_pad, cx<R> (&s)[12]) {
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf((float)s[k].r), fabsf((float)s[k].i)));
  float inv = m > 0.f ? 1.0f / m : 0.f;
  int4* p = (int4*)base;
  float* sc = (float*)((char*)base + (size_t)Vh_pad * 48);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    int4 v;
    __half2* h = reinterpret_cast<__half2*>(&v);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      h[j] = __floats2half2_rn((float)s[4 * k + j].r * inv, (float)s[4 * k + j].i * inv);
      if constexpr (KEEP) {
        const float2 f = __half22float2(h[j]);
        s[4 * k + j] = mk<R>((R)(f.x * m), (R)(f.y * m));
      }
    }
    p[sbi(cb, k, 3)] = v;
  }
  sc[cb] = m;
}

template <int P, typename R>
__device__ __forceinline__ void store_spinor(void* base, int cb, int Vh_pad, const cx<R> (&s)[12]) {
  if constexpr (P == WD_F64) {
    double2* p = (double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) p[sbi(cb, k, 12)] = make_double2((double)s[k].r, (double)s[k].i);
  } else if constexpr (P == WD_F32) {
    float4* p = (float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++)
      p[sbi(cb, k, 6)] = make_float4((float)s[2 * k].r, (float)s[2 * k].i,
                                     (float)s[2 * k + 1].r, (float)s[2 * k + 1].i);
  } else {
    store_spinor_f16<R, false>(base, cb, Vh_pad, const_cast<cx<R>(&)[12]>(s));
  }
}

// ---------------------------------------------------------------------------
// packed gauge formats: 8 regions (mu, parity of the base site), region
// r = 2*mu + par holds Vh_pad sites.
//   (F64,18): 9 double2 (row-major entries)     (F64,12): 6 double2 (rows 0,1)
//   (F32,18): 9 float2                           (F32,12): 3 float4 (rows 0,1)
//   (F16,12): 1 int4 (U00 U01 U02 U10 as half2) in the first 8 regions, then
//             1 int2 (U11 U12) in 8 more regions
// ---------------------------------------------------------------------------

inline size_t link_bytes(int prec, int recon) {
  if (prec == WD_F64) return recon == 18 ? 144 : 96;
  if (prec == WD_F32) return recon == 18 ? 72 : 48;
  if (prec == WD_F16 && recon == 12) return 24;
  return 0;
}

inline size_t gauge_bytes(const Geom& g, int prec, int recon) {
  return round_up((size_t)8 * g.Vh_pad * link_bytes(prec, recon), 256);
}

// rebuild row 2 of an SU(3) matrix from rows 0 and 1: row2 = conj(row0 x row1)
template <typename R>
__device__ __forceinline__ void reconstruct_row2(cx<R> (&u)[9]) {
  u[6] = conj_cross(u[1], u[5], u[2], u[4]);
  u[7] = conj_cross(u[2], u[3], u[0], u[5]);
  u[8] = conj_cross(u[0], u[4], u[1], u[3]);
}

template <int P, int RC, typename R>
__device__ __forceinline__ void load_link(cx<R> (&u)[9], const void* gauge, int region, int cb,
                                          int Vh_pad) {
  if constexpr (P == WD_F64) {
    constexpr int NC = RC == 18 ? 9 : 6;
    const double2* p = (const double2*)gauge + (size_t)region * Vh_pad * NC;
#pragma unroll
    for (int k = 0; k < NC; k++) {
      double2 v = __ldg(p + sbi(cb, k, NC));
      u[k] = mk<R>((R)v.x, (R)v.y);
    }
  } else if constexpr (P == WD_F32) {
    if constexpr (RC == 18) {
      const float2* p = (const float2*)gauge + (size_t)region * Vh_pad * 9;
#pragma unroll
      for (int k = 0; k < 9; k++) {
        float2 v = __ldg(p + sbi(cb, k, 9));
        u[k] = mk<R>((R)v.x, (R)v.y);
      }
    } else {
      const float4* p = (const float4*)gauge + (size_t)region * Vh_pad * 3;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        float4 v = __ldg(p + sbi(cb, k, 3));
        u[2 * k] = mk<R>((R)v.x, (R)v.y);
        u[2 * k + 1] = mk<R>((R)v.z, (R)v.w);
      }
    }
  } else {
    const int4* pa = (const int4*)gauge + (size_t)region * Vh_pad;
    const int2* pb = (const int2*)((const char*)gauge + (size_t)8 * Vh_pad * 16) + (size_t)region * Vh_pad;
    int4 a = __ldg(pa + sbi(cb, 0, 1));
    int2 b = __ldg(pb + sbi(cb, 0, 1));
    const __half2* ha = reinterpret_cast<const __half2*>(&a);
    const __half2* hb = reinterpret_cast<const __half2*>(&b);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float2 f = __half22float2(ha[j]);
      u[j] = mk<R>((R)f.x, (R)f.y);
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
      float2 f = __half22float2(hb[j]);
      u[4 + j] = mk<R>((R)f.x, (R)f.y);
    }
  }
  if constexpr (RC == 12) reconstruct_row2(u);
}

// ---------------------------------------------------------------------------
// deterministic FP64 reduction: block tree -> per-block partials -> the last
// block to finish sums the partials in a fixed order and calls `fin`.
// ---------------------------------------------------------------------------

struct RedScratch {
  double* partials;    // >= gridDim.x * N doubles
  unsigned* counter;   // zero between kernels; reset by the last block
};

// Sum over the BS threads of a block (1-, 2- or 3-dimensional; warps are
// taken in linear thread order), in the type T.  The total is in every
// thread of warp 0.
template <int N, int BS, typename T = double>
__device__ __forceinline__ void block_sum(T (&v)[N], T* smem /* N * BS/32 */) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < N; j++) {
    T t = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    v[j] = t;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < N; j++) smem[j * (BS / 32) + warp] = v[j];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < N; j++) {
      T t = lane < BS / 32 ? smem[j * (BS / 32) + lane] : (T)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[j] = t;
    }
  }
}

// The block's share of a grid sum, without the cross-block step: the block
// sums v in T and thread 0 stores its N totals as FP64 partials.  A separate
// launch that follows the kernel in its stream (sum_block_partials) adds the
// partials in block order.  Unlike grid_reduce, no block waits for an atomic
// round trip before it exits.
template <int N, int BS, typename T>
__device__ __forceinline__ void block_partials(T (&v)[N], double* partials) {
  __shared__ T smem[N * (BS / 32)];
  block_sum<N, BS, T>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < N; j++) partials[(size_t)blockIdx.x * N + j] = (double)v[j];
  }
}

// Returns true in every thread of the last block; there `tot` holds the grid
// total in thread 0 (and all threads of warp 0).  The block sums in T (the
// kernel's working precision), the block partials in FP64.
template <int N, int BS, typename T = double>
__device__ __forceinline__ bool grid_reduce(T (&v)[N], RedScratch rs, double (&tot)[N]) {
  __shared__ T tsmem[N * (BS / 32)];
  __shared__ double smem[N * (BS / 32)];
  __shared__ bool last;
  block_sum<N, BS, T>(v, tsmem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < N; j++) rs.partials[(size_t)blockIdx.x * N + j] = (double)v[j];
    // one acquire-release arrival: it orders the partials written above
    // before it for the last block, and that block's reads after it
    unsigned t;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(t) : "l"(rs.counter) : "memory");
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // CH independent chains per thread keep CH loads of the partials in flight
  // (a single chain waits one L2 round trip per partial); the chains are
  // combined in a fixed order, so the sum does not depend on scheduling
  constexpr int CH = N == 1 ? 8 : (N <= 4 ? 4 : 1);
  double part[CH][N];
#pragma unroll
  for (int c = 0; c < CH; c++)
#pragma unroll
    for (int j = 0; j < N; j++) part[c][j] = 0.0;
  int b = threadIdx.x;
  for (; b + (CH - 1) * BS < (int)gridDim.x; b += CH * BS) {
#pragma unroll
    for (int c = 0; c < CH; c++)
#pragma unroll
      for (int j = 0; j < N; j++) part[c][j] += __ldcg(rs.partials + (size_t)(b + c * BS) * N + j);
  }
  for (; b < (int)gridDim.x; b += BS) {
#pragma unroll
    for (int j = 0; j < N; j++) part[0][j] += __ldcg(rs.partials + (size_t)b * N + j);
  }
  double acc[N];
#pragma unroll
  for (int j = 0; j < N; j++) {
    double t = part[0][j];
#pragma unroll
    for (int c = 1; c < CH; c++) t += part[c][j];
    acc[j] = t;
  }
  __syncthreads();
  block_sum<N, BS>(acc, smem);
#pragma unroll
  for (int j = 0; j < N; j++) tot[j] = acc[j];
  if (threadIdx.x == 0) *rs.counter = 0u;
  return true;
}

}  // namespace wd
