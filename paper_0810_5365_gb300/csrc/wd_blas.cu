// Field layout conversions (canonical FP64 <-> packed, precision changes) and
// the BLAS-like vector kernels with FP64 reductions.  The paper's solver is a
// sequence of kernels: Dslash, a dot product whose global sum is done on the
// GPU in double precision by parallel reduction, and BLAS-like updates
// (section "Wilson inverter: Main features").  Reductions here are two-level
// and deterministic: fixed grid, fixed tree inside a block, and a fixed-order
// sum of the per-block partials, either by the last block to finish
// (grid_reduce: wd_norm2, wd_cdot) or by a one-CTA launch that follows the
// kernel in its stream (sum_block_partials: the fused norms of the solvers).
#include "wd_internal.h"

namespace wd {

// ---------------------------------------------------------------------------
// library state shared by the translation units
// ---------------------------------------------------------------------------

State& state() {
  static State s;
  return s;
}

int num_sms() {
  State& s = state();
  if (s.num_sms == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    s.num_sms = n > 0 ? n : 1;
  }
  return s.num_sms;
}

int blas_grid(long long n, int bs) {
  long long need = (n + bs - 1) / bs;
  long long cap = (long long)num_sms() * 8;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

cudaError_t ensure_scratch(size_t doubles) {
  State& s = state();
  if (!s.counter) {
    cudaError_t e = cudaMalloc(&s.counter, 256);
    if (e != cudaSuccess) return e;
    e = cudaMemset(s.counter, 0, 256);
    if (e != cudaSuccess) return e;
  }
  if (doubles <= s.partials_cap) return cudaSuccess;
  size_t cap = doubles < 65536 ? 65536 : doubles;
  if (s.partials) {
    cudaDeviceSynchronize();
    cudaFree(s.partials);
    s.partials = nullptr;
    s.partials_cap = 0;
  }
  cudaError_t e = cudaMalloc(&s.partials, cap * sizeof(double));
  if (e != cudaSuccess) return e;
  s.partials_cap = cap;
  return cudaSuccess;
}

cudaError_t device_flag(int** flag, cudaStream_t st) {
  State& s = state();
  if (!s.dev_flag) {
    cudaError_t e = cudaMalloc(&s.dev_flag, 256);
    if (e != cudaSuccess) return e;
  }
  *flag = s.dev_flag;
  return cudaMemsetAsync(s.dev_flag, 0, sizeof(int), st);
}

// The cross-block step of block_partials, in the same fixed order as the
// last block of grid_reduce: CH chains per thread over the partials, combined
// in order, then a block sum.
template <int N>
__global__ void __launch_bounds__(256) sum_blocks_kernel(const double* __restrict__ partials,
                                                         int nblocks, SumOut out) {
  constexpr int BS = 256;
  constexpr int CH = N == 1 ? 8 : 4;
  __shared__ double smem[N * (BS / 32)];
  pdl_begin();
  double part[CH][N];
#pragma unroll
  for (int c = 0; c < CH; c++)
#pragma unroll
    for (int j = 0; j < N; j++) part[c][j] = 0.0;
  int b = threadIdx.x;
  for (; b + (CH - 1) * BS < nblocks; b += CH * BS) {
#pragma unroll
    for (int c = 0; c < CH; c++)
#pragma unroll
      for (int j = 0; j < N; j++) part[c][j] += __ldcg(partials + (size_t)(b + c * BS) * N + j);
  }
  for (; b < nblocks; b += BS) {
#pragma unroll
    for (int j = 0; j < N; j++) part[0][j] += __ldcg(partials + (size_t)b * N + j);
  }
  double acc[N];
#pragma unroll
  for (int j = 0; j < N; j++) {
    double t = part[0][j];
#pragma unroll
    for (int c = 1; c < CH; c++) t += part[c][j];
    acc[j] = t;
  }
  block_sum<N, BS>(acc, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < N; j++)
      if (out.p[j]) *out.p[j] = acc[j];
  }
}

cudaError_t sum_block_partials(int n, const double* partials, int nblocks, SumOut out,
                               cudaStream_t st) {
  switch (n) {
    case 1: return launch_pdl(sum_blocks_kernel<1>, dim3(1), dim3(256), st, partials, nblocks, out);
    case 2: return launch_pdl(sum_blocks_kernel<2>, dim3(1), dim3(256), st, partials, nblocks, out);
    case 3: return launch_pdl(sum_blocks_kernel<3>, dim3(1), dim3(256), st, partials, nblocks, out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t sum_block_partials(int n, const double* partials, int nblocks, double* out,
                               cudaStream_t st) {
  SumOut o = {{out, n > 1 ? out + 1 : nullptr, n > 2 ? out + 2 : nullptr}};
  return sum_block_partials(n, partials, nblocks, o, st);
}

RedScratch scratch() {
  RedScratch r;
  r.partials = state().partials;
  r.counter = state().counter;
  return r;
}

// ---------------------------------------------------------------------------
// canonical <-> packed spinors
// ---------------------------------------------------------------------------

__device__ __forceinline__ int lex_parity(int i, const Geom& g) {
  int x0 = i % g.L[0];
  int r = i / g.L[0];
  int x1 = r % g.L[1];
  r /= g.L[1];
  int x2 = r % g.L[2];
  int x3 = r / g.L[2];
  return (x0 + x1 + x2 + x3) & 1;
}

// src: canonical complex double [n][12]; half layout (full = 0) indexes by cb,
// full layout (full = 1) by lexicographic site.
template <int P>
__global__ void pack_spinor_kernel(char* dst, const double2* __restrict__ src, Geom g, int full,
                                   size_t half_bytes) {
  long long n = full ? 2LL * g.Vh : g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int cb = full ? (int)(i >> 1) : (int)i;
    int par = full ? lex_parity((int)i, g) : 0;
    cx<double> s[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = src[i * 12 + k];
      s[k] = mk<double>(v.x, v.y);
    }
    store_spinor<P, double>(dst + par * half_bytes, cb, g.Vh_pad, s);
  }
}

template <int P>
__global__ void unpack_spinor_kernel(double2* dst, const char* __restrict__ src, Geom g, int full,
                                     size_t half_bytes) {
  long long n = full ? 2LL * g.Vh : g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int cb = full ? (int)(i >> 1) : (int)i;
    int par = full ? lex_parity((int)i, g) : 0;
    cx<double> s[12];
    load_spinor_rw<P, double>(s, src + par * half_bytes, cb, g.Vh_pad);
#pragma unroll
    for (int k = 0; k < 12; k++) dst[i * 12 + k] = make_double2(s[k].r, s[k].i);
  }
}

#define WD_PREC_SWITCH(prec, F, ...)                  \
  switch (prec) {                                      \
    case WD_F64: F<WD_F64><<<__VA_ARGS__; break;       \
    case WD_F32: F<WD_F32><<<__VA_ARGS__; break;       \
    case WD_F16: F<WD_F16><<<__VA_ARGS__; break;       \
    default: return cudaErrorInvalidValue;             \
  }

cudaError_t pack_spinor(void* dst, const double* src, const Geom& g, int parity, int prec,
                        cudaStream_t st) {
  int full = parity == WD_FULL;
  long long n = full ? 2LL * g.Vh : g.Vh;
  int grid = blas_grid(n, 256);
  size_t hb = spinor_half_bytes(g, prec);
  WD_PREC_SWITCH(prec, pack_spinor_kernel, grid, 256, 0, st>>>((char*)dst, (const double2*)src, g,
                                                                full, hb))
  return cudaGetLastError();
}

cudaError_t unpack_spinor(double* dst, const void* src, const Geom& g, int parity, int prec,
                          cudaStream_t st) {
  int full = parity == WD_FULL;
  long long n = full ? 2LL * g.Vh : g.Vh;
  int grid = blas_grid(n, 256);
  size_t hb = spinor_half_bytes(g, prec);
  WD_PREC_SWITCH(prec, unpack_spinor_kernel, grid, 256, 0, st>>>((double2*)dst, (const char*)src,
                                                                  g, full, hb))
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gauge packing
// ---------------------------------------------------------------------------

template <int P, int RC>
__device__ __forceinline__ void store_link(char* gauge, int region, int cb, int Vh_pad,
                                           const cx<double> (&u)[9]) {
  if constexpr (P == WD_F64) {
    constexpr int NC = RC == 18 ? 9 : 6;
    double2* p = (double2*)gauge + (size_t)region * Vh_pad * NC;
#pragma unroll
    for (int k = 0; k < NC; k++) p[sbi(cb, k, NC)] = make_double2(u[k].r, u[k].i);
  } else if constexpr (P == WD_F32) {
    if constexpr (RC == 18) {
      float2* p = (float2*)gauge + (size_t)region * Vh_pad * 9;
#pragma unroll
      for (int k = 0; k < 9; k++) p[sbi(cb, k, 9)] = make_float2((float)u[k].r, (float)u[k].i);
    } else {
      float4* p = (float4*)gauge + (size_t)region * Vh_pad * 3;
#pragma unroll
      for (int k = 0; k < 3; k++)
        p[sbi(cb, k, 3)] = make_float4((float)u[2 * k].r, (float)u[2 * k].i,
                                       (float)u[2 * k + 1].r, (float)u[2 * k + 1].i);
    }
  } else {
    int4* pa = (int4*)gauge + (size_t)region * Vh_pad;
    int2* pb = (int2*)(gauge + (size_t)8 * Vh_pad * 16) + (size_t)region * Vh_pad;
    int4 a;
    int2 b;
    __half2* ha = reinterpret_cast<__half2*>(&a);
    __half2* hb = reinterpret_cast<__half2*>(&b);
#pragma unroll
    for (int j = 0; j < 4; j++) ha[j] = __floats2half2_rn((float)u[j].r, (float)u[j].i);
#pragma unroll
    for (int j = 0; j < 2; j++) hb[j] = __floats2half2_rn((float)u[4 + j].r, (float)u[4 + j].i);
    pa[sbi(cb, 0, 1)] = a;
    pb[sbi(cb, 0, 1)] = b;
  }
}

// src: canonical [4][V][3][3] complex double; one thread per (mu, site)
template <int P, int RC>
__global__ void pack_gauge_kernel(char* dst, const double2* __restrict__ src, Geom g) {
  long long V = 2LL * g.Vh;
  long long n = 4 * V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int mu = (int)(t / V);
    int i = (int)(t - mu * V);
    int par = lex_parity(i, g);
    cx<double> u[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      double2 v = src[t * 9 + k];
      u[k] = mk<double>(v.x, v.y);
    }
    store_link<P, RC>(dst, 2 * mu + par, i >> 1, g.Vh_pad, u);
  }
}

cudaError_t pack_gauge(void* dst, const double* src, const Geom& g, int prec, int recon,
                       cudaStream_t st) {
  int grid = blas_grid(8LL * g.Vh, 256);
  const double2* s = (const double2*)src;
  char* d = (char*)dst;
  if (prec == WD_F64 && recon == 18) pack_gauge_kernel<WD_F64, 18><<<grid, 256, 0, st>>>(d, s, g);
  else if (prec == WD_F64 && recon == 12) pack_gauge_kernel<WD_F64, 12><<<grid, 256, 0, st>>>(d, s, g);
  else if (prec == WD_F32 && recon == 18) pack_gauge_kernel<WD_F32, 18><<<grid, 256, 0, st>>>(d, s, g);
  else if (prec == WD_F32 && recon == 12) pack_gauge_kernel<WD_F32, 12><<<grid, 256, 0, st>>>(d, s, g);
  else if (prec == WD_F16 && recon == 12) pack_gauge_kernel<WD_F16, 12><<<grid, 256, 0, st>>>(d, s, g);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// precision conversion, BLAS and reductions (nh halves of Vh sites each)
// ---------------------------------------------------------------------------

template <int PD, int PS>
__global__ void convert_kernel(char* dst, const char* __restrict__ src, Geom g, int nh,
                               size_t dhb, size_t shb) {
  long long n = (long long)nh * g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    using R = typename std::conditional<PD == WD_F64 || PS == WD_F64, double, float>::type;
    cx<R> s[12];
    load_spinor_rw<PS, R>(s, src + h * shb, cb, g.Vh_pad);
    store_spinor<PD, R>(dst + h * dhb, cb, g.Vh_pad, s);
  }
}

cudaError_t convert_spinor(void* dst, int dprec, const void* src, int sprec, const Geom& g, int nh,
                           cudaStream_t st) {
  int grid = blas_grid((long long)nh * g.Vh, 256);
  size_t dhb = spinor_half_bytes(g, dprec), shb = spinor_half_bytes(g, sprec);
  char* d = (char*)dst;
  const char* s = (const char*)src;
#define WD_CV(A, B)                                                                 \
  if (dprec == A && sprec == B) {                                                   \
    convert_kernel<A, B><<<grid, 256, 0, st>>>(d, s, g, nh, dhb, shb);              \
    return cudaGetLastError();                                                      \
  }
  WD_CV(WD_F64, WD_F64) WD_CV(WD_F64, WD_F32) WD_CV(WD_F64, WD_F16)
  WD_CV(WD_F32, WD_F64) WD_CV(WD_F32, WD_F32) WD_CV(WD_F32, WD_F16)
  WD_CV(WD_F16, WD_F64) WD_CV(WD_F16, WD_F32) WD_CV(WD_F16, WD_F16)
#undef WD_CV
  return cudaErrorInvalidValue;
}

template <int P, int BS>
__global__ void __launch_bounds__(BS) norm2_kernel(double* res, const char* __restrict__ x, Geom g,
                                                   int nh, size_t hb, RedScratch rs) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  long long n = (long long)nh * g.Vh;
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)BS + threadIdx.x; i < n; i += (long long)gridDim.x * BS) {
    int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<R> s[12];
    load_spinor_rw<P, R>(s, x + h * hb, cb, g.Vh_pad);
    acc[0] += site_norm2(s);
  }
  double tot[1];
  if (grid_reduce<1, BS>(acc, rs, tot) && threadIdx.x == 0) res[0] = tot[0];
}

template <int P, int BS>
__global__ void __launch_bounds__(BS) cdot_kernel(double* res, const char* __restrict__ x,
                                                  const char* __restrict__ y, Geom g, int nh,
                                                  size_t hb, RedScratch rs) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  long long n = (long long)nh * g.Vh;
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)BS + threadIdx.x; i < n; i += (long long)gridDim.x * BS) {
    int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<R> a[12], b[12];
    load_spinor_rw<P, R>(a, x + h * hb, cb, g.Vh_pad);
    load_spinor_rw<P, R>(b, y + h * hb, cb, g.Vh_pad);
    site_cdot(a, b, acc[0], acc[1]);
  }
  double tot[2];
  if (grid_reduce<2, BS>(acc, rs, tot) && threadIdx.x == 0) {
    res[0] = tot[0];
    res[1] = tot[1];
  }
}

template <int P>
__global__ void axpby_kernel(double a, const char* __restrict__ x, double b, char* y, Geom g,
                             int nh, size_t hb) {
  using R = typename std::conditional<P == WD_F64, double, float>::type;
  long long n = (long long)nh * g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<R> u[12], v[12];
    load_spinor_rw<P, R>(u, x + h * hb, cb, g.Vh_pad);
    if (b != 0.0) {
      load_spinor_rw<P, R>(v, y + h * hb, cb, g.Vh_pad);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        v[k].r = (R)a * u[k].r + (R)b * v[k].r;
        v[k].i = (R)a * u[k].i + (R)b * v[k].i;
      }
    } else {
      // b = 0: y is output only and never read (BLAS convention), so an
      // uninitialised y cannot leak NaN or Inf through 0 * y
#pragma unroll
      for (int k = 0; k < 12; k++) v[k] = mk<R>((R)a * u[k].r, (R)a * u[k].i);
    }
    store_spinor<P, R>(y + h * hb, cb, g.Vh_pad, v);
  }
}

constexpr int RED_BS = 256;

cudaError_t norm2(double* res, const void* x, const Geom& g, int prec, int nh, cudaStream_t st) {
  int grid = blas_grid((long long)nh * g.Vh, RED_BS);
  cudaError_t e = ensure_scratch((size_t)grid * 2);
  if (e != cudaSuccess) return e;
  size_t hb = spinor_half_bytes(g, prec);
  RedScratch rs = scratch();
  switch (prec) {
    case WD_F64: norm2_kernel<WD_F64, RED_BS><<<grid, RED_BS, 0, st>>>(res, (const char*)x, g, nh, hb, rs); break;
    case WD_F32: norm2_kernel<WD_F32, RED_BS><<<grid, RED_BS, 0, st>>>(res, (const char*)x, g, nh, hb, rs); break;
    case WD_F16: norm2_kernel<WD_F16, RED_BS><<<grid, RED_BS, 0, st>>>(res, (const char*)x, g, nh, hb, rs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t cdot(double* res, const void* x, const void* y, const Geom& g, int prec, int nh,
                 cudaStream_t st) {
  int grid = blas_grid((long long)nh * g.Vh, RED_BS);
  cudaError_t e = ensure_scratch((size_t)grid * 2);
  if (e != cudaSuccess) return e;
  size_t hb = spinor_half_bytes(g, prec);
  RedScratch rs = scratch();
  const char* a = (const char*)x;
  const char* b = (const char*)y;
  switch (prec) {
    case WD_F64: cdot_kernel<WD_F64, RED_BS><<<grid, RED_BS, 0, st>>>(res, a, b, g, nh, hb, rs); break;
    case WD_F32: cdot_kernel<WD_F32, RED_BS><<<grid, RED_BS, 0, st>>>(res, a, b, g, nh, hb, rs); break;
    case WD_F16: cdot_kernel<WD_F16, RED_BS><<<grid, RED_BS, 0, st>>>(res, a, b, g, nh, hb, rs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t axpby(double a, const void* x, double b, void* y, const Geom& g, int prec, int nh,
                  cudaStream_t st) {
  int grid = blas_grid((long long)nh * g.Vh, 256);
  size_t hb = spinor_half_bytes(g, prec);
  WD_PREC_SWITCH(prec, axpby_kernel, grid, 256, 0, st>>>(a, (const char*)x, b, (char*)y, g, nh, hb))
  return cudaGetLastError();
}

}  // namespace wd
