// Learned gauge-covariant preconditioner: a three-layer linear network of the
// nearest-neighbour layers of wd_nn.cuh (4 -> 8 -> 8 -> 4 spin-like channels
// per colour, i.e. 12 -> 24 -> 24 -> 12 complex channels per site), trained
// on pairs (b = D x, x) drawn on the GPU to minimise ||N(b) - x||^2, and used
// as the preconditioner of flexible GCR.  None of this is in the paper; it
// sits on top of the paper's operator and kernels.
#include <chrono>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "wd_nn.cuh"

namespace wd {

// parameter layout: layer l has 9 x COUT_l x CIN_l complex weights, stored
// [d][o][i][re, im], layers back to back
constexpr int NN_C[4] = {4, 8, 8, 4};
constexpr int nn_layer_floats(int l) { return 9 * NN_C[l + 1] * NN_C[l] * 2; }
constexpr int nn_layer_offset(int l) {
  return l == 0 ? 0 : nn_layer_offset(l - 1) + nn_layer_floats(l - 1);
}
constexpr int NN_PARAMS = nn_layer_offset(3);  // 2304 floats

// ---------------------------------------------------------------------------
// layer launch
// ---------------------------------------------------------------------------

// persistent grid: as many CTAs as fit on the SMs at once (at most 8 per SM,
// the 512 TMEM columns / 64 per CTA), never more than there are tiles
template <int CIN, int COUT, bool BIN = false, bool BOUT = false>
static cudaError_t launch_layer(const NnLayerArgs& A, int ntiles, cudaStream_t st) {
  // residency from the kernel's own register and shared-memory footprint
  // (registers are allocated per warp in units of 256)
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, nn_layer_kernel<CIN, COUT, BIN, BOUT>);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int regs_sm = 0, smem_sm = 0, thr_sm = 0;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs_sm / (warp_regs * (NN_THREADS / 32));
    const int by_smem = smem_sm / ((int)fa.sharedSizeBytes + 1024);
    const int by_thr = thr_sm / NN_THREADS;
    int n = by_regs < by_smem ? by_regs : by_smem;
    n = n < by_thr ? n : by_thr;
    n = n < 1 ? 1 : (n > 8 ? 8 : n);
    // ask for a shared-memory carveout that holds all n CTAs
    const int pct = (int)((100LL * n * ((int)fa.sharedSizeBytes + 1024) + smem_sm - 1) / smem_sm);
    e = cudaFuncSetAttribute(nn_layer_kernel<CIN, COUT, BIN, BOUT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, pct < 100 ? pct : 100);
    if (e != cudaSuccess) return e;
    per_sm = n;
  }
  const int cap = num_sms() * per_sm;
  const int grid = ntiles < cap ? ntiles : cap;
  nn_layer_kernel<CIN, COUT, BIN, BOUT><<<grid, NN_THREADS, 0, st>>>(A, ntiles);
  return cudaGetLastError();
}

// the one-thread-per-site inference kernel, with its residency computed the
// same way
// (returns cudaErrorNotReady, launching nothing, when ntiles is below two
// waves of its CTAs: a 4-warp CTA takes twice as long per tile as the
// two-thread kernel's 8-warp one, so with one or two tiles per CTA the
// two-thread kernel is the faster)
template <int CIN, int COUT, bool BIN, bool BOUT>
static cudaError_t launch_infer(const NnLayerArgs& A, int ntiles, cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, nn_infer_kernel<CIN, COUT, BIN, BOUT>);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int regs_sm = 0, smem_sm = 0, thr_sm = 0;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs_sm / (warp_regs * (NN_TILE / 32));
    const int by_smem = smem_sm / ((int)fa.sharedSizeBytes + 1024);
    const int by_thr = thr_sm / NN_TILE;
    int n = by_regs < by_smem ? by_regs : by_smem;
    n = n < by_thr ? n : by_thr;
    // (at most 8: eight CTAs fill the 512 TMEM columns of an SM)
    n = n < 1 ? 1 : (n > 8 ? 8 : n);
    const int pct = (int)((100LL * n * ((int)fa.sharedSizeBytes + 1024) + smem_sm - 1) / smem_sm);
    e = cudaFuncSetAttribute(nn_infer_kernel<CIN, COUT, BIN, BOUT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, pct < 100 ? pct : 100);
    if (e != cudaSuccess) return e;
    per_sm = n;
  }
  const int cap = num_sms() * per_sm;
  if (ntiles < 2 * cap) return cudaErrorNotReady;
  nn_infer_kernel<CIN, COUT, BIN, BOUT><<<cap, NN_TILE, 0, st>>>(A, ntiles);
  return cudaGetLastError();
}

#ifndef WD_NN_INFER1
#define WD_NN_INFER1 1  // BF16 inference layers: the one-thread-per-site kernel
#endif

// out_parity: -1 both parities, else only that one; zero_in: the parity of
// the input known to vanish (never read), or -1
static cudaError_t nn_layer(int cin, int cout, const Geom& g, const void* gauge, const void* in,
                            void* out, const float* w, int* err, cudaStream_t st,
                            int out_parity = -1, int zero_in = -1) {
  NnLayerArgs A;
  A.g = g;
  A.gauge = gauge;
  A.in = (const char*)in;
  A.out = (char*)out;
  A.in_half = nn_half_bytes(g.Vh_pad, cin);
  A.out_half = nn_half_bytes(g.Vh_pad, cout);
  A.w = w;
  A.err = err;
  A.p0 = out_parity < 0 ? 0 : out_parity;
  A.np = out_parity < 0 ? 2 : 1;
  A.zero_in = zero_in;
  const int ntiles = A.np * ((g.Vh + NN_TILE - 1) / NN_TILE);
  if (cin == 4 && cout == 8) return launch_layer<4, 8>(A, ntiles, st);
  if (cin == 8 && cout == 8) return launch_layer<8, 8>(A, ntiles, st);
  if (cin == 8 && cout == 4) return launch_layer<8, 4>(A, ntiles, st);
  if (cin == 4 && cout == 4) return launch_layer<4, 4>(A, ntiles, st);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// weight gradient: G_d[o][i] = sum_{x, a} delta(x)[o][a] conj((T_d phi)(x)[i][a])
// (the tensor-core kernel below writes one partial gradient per CTA; this
// sums them in CTA order)
// ---------------------------------------------------------------------------

// out[j] (+)= sum_t partials[t][j], t in order
__global__ void nn_sum_tiles(const float* __restrict__ partials, int ntiles, int n, float* out,
                             int accumulate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int t = 0; t < ntiles; t++) s += (double)partials[(size_t)t * n + j];
  out[j] = accumulate ? out[j] + (float)s : (float)s;
}

// ---------------------------------------------------------------------------
// weight gradient on the tensor cores: for all nine directions at once,
//   G^T[d C_in + i][2o + part] = sum_{x, a} (T_d phi)[i][a] x delta-row,
// with the real form of the complex product conj-contracted over (site,
// colour): the A rows are the transported input channels [t_r | t_i] (9 C_in
// of the M = 128 rows, the rest zero), the B rows are [delta_r | delta_i] for
// Re G and [delta_i | -delta_r] for Im G (2 C_out of N = 16 rows).  K runs over
// (part, colour, site) of 32-site blocks: 192 = 12 chunks of 16 per block.
// Each persistent CTA accumulates its blocks in TMEM (FP32), writes its
// partial gradient, and the partials are summed over CTAs in a fixed order.
// ---------------------------------------------------------------------------

constexpr int WG_SITES = 32;                    // sites per K block
constexpr int WG_KCH = 2 * 3 * WG_SITES / 16;   // K chunks of 16 per block
constexpr uint32_t WG_ACH = 128 * 16 * 2;       // one A chunk (M = 128 rows), bytes
constexpr uint32_t WG_BCH = 16 * 16 * 2;        // one B chunk (N = 16 rows), bytes
constexpr uint32_t WG_BUF = WG_KCH * (WG_ACH + WG_BCH);
constexpr int WG_THREADS = 256;

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS) nn_wgrad_tc_kernel(const NnLayerArgs A,
                                                                 const char* __restrict__ delta,
                                                                 size_t delta_half, int nblocks,
                                                                 float* partials) {
  extern __shared__ __align__(128) unsigned char wg_smem[];  // 2 buffers of WG_BUF
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geom& g = A.g;
  constexpr int NV = NN_NDIR * COUT * CIN * 2;
  // rows that are never written (A rows >= 9 CIN, B rows >= 2 COUT) stay zero
  for (uint32_t e = tid; e < 2 * WG_BUF / 16; e += WG_THREADS)
    reinterpret_cast<int4*>(wg_smem)[e] = make_int4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 32);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = make_idesc_bf16(128, 16);
  const int bpp = (g.Vh + WG_SITES - 1) / WG_SITES;  // blocks per parity
  // work split of the 8 warps: CIN = 8: warps w and w + 4 transport channels
  // 0-3 and 4-7 of directions w, w + 4, w + 8; CIN = 4: warps 0-3 transport
  // directions w, w + 4, w + 8 and warps 4-7 stage the delta rows
  constexpr bool SPLIT = CIN == 8;
  const int dw = warp & 3;
  const int c0 = SPLIT ? 4 * (warp >> 2) : 0;
  const bool transports = SPLIT || warp < 4;
  bool ok = true;
  uint32_t G = 0;  // blocks issued by this CTA

  for (int blk = blockIdx.x; blk < nblocks; blk += gridDim.x, G++) {
    const uint32_t buf = G & 1u;
    unsigned char* sa = wg_smem + buf * WG_BUF;
    unsigned char* sb = sa + WG_KCH * WG_ACH;
    if (G >= 2) ok = mbar_wait_bounded(&bar[buf], ((G - 2) >> 1) & 1u, NN_SPIN_LIMIT) && ok;
    const int p = blk / bpp;
    const int cb = (blk - p * bpp) * WG_SITES + lane;
    const bool valid = cb < g.Vh;
    if (transports) {
      int nb[NN_NDIR];
      int x3 = 0;
      if (valid) nn_nbr(nb, x3, cb, p, g);
      for (int d = dw; d < NN_NDIR; d += 4) {
        cx<float> t[12];
        if (valid) {
          nn_transport4<CIN>(t, A, d, p, cb, nb[d], x3, c0);
        } else {
#pragma unroll
          for (int k = 0; k < 12; k++) t[k] = mk<float>(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
#pragma unroll
          for (int a = 0; a < 3; a++) {
#pragma unroll
            for (int part = 0; part < 2; part++) {
              const int kp = (part * 3 + a) * WG_SITES + lane;
              const float v = part ? t[i * 3 + a].i : t[i * 3 + a].r;
              *(__nv_bfloat16*)(sa + (kp >> 4) * WG_ACH +
                                kmajor_offset(d * CIN + c0 + i, kp & 15, 16)) =
                  __float2bfloat16_rn(v);
            }
          }
        }
      }
    }
    // B: the delta rows of these sites, output channels spread over the warps
    // that do not transport (CIN = 4) or over all warps (CIN = 8)
    {
      constexpr int NW = SPLIT ? 8 : 4;
      const int w0 = SPLIT ? warp : warp - 4;
      if (w0 >= 0) {
        for (int o = w0; o < COUT; o += NW) {
          cx<float> dl[3];
          if (valid) {
            const float4* src = (const float4*)(delta + p * delta_half);
            constexpr int NG = 3 * COUT / 2;
            // complex index o*3 + a lives in group (o*3 + a) / 2, half (o*3 + a) % 2
#pragma unroll
            for (int a = 0; a < 3; a++) {
              const int ci = o * 3 + a;
              const float4 q = __ldg(src + sbi(cb, ci >> 1, NG));
              dl[a] = (ci & 1) ? mk<float>(q.z, q.w) : mk<float>(q.x, q.y);
            }
          } else {
#pragma unroll
            for (int a = 0; a < 3; a++) dl[a] = mk<float>(0.f, 0.f);
          }
#pragma unroll
          for (int a = 0; a < 3; a++) {
            const cx<float> v = dl[a];
            const int k0 = a * WG_SITES + lane, k1 = (3 + a) * WG_SITES + lane;
            // Re G row: [delta_r | delta_i] ; Im G row: [delta_i | -delta_r]
            *(__nv_bfloat16*)(sb + (k0 >> 4) * WG_BCH + kmajor_offset(2 * o, k0 & 15, 16)) =
                __float2bfloat16_rn(v.r);
            *(__nv_bfloat16*)(sb + (k1 >> 4) * WG_BCH + kmajor_offset(2 * o, k1 & 15, 16)) =
                __float2bfloat16_rn(v.i);
            *(__nv_bfloat16*)(sb + (k0 >> 4) * WG_BCH + kmajor_offset(2 * o + 1, k0 & 15, 16)) =
                __float2bfloat16_rn(v.i);
            *(__nv_bfloat16*)(sb + (k1 >> 4) * WG_BCH + kmajor_offset(2 * o + 1, k1 & 15, 16)) =
                __float2bfloat16_rn(-v.r);
          }
        }
      }
    }
      fence_smem_to_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      for (int kc = 0; kc < WG_KCH; kc++) {
        const uint64_t ad = make_smem_desc(smem_u32(sa + kc * WG_ACH), 128, 256);
        const uint64_t bd = make_smem_desc(smem_u32(sb + kc * WG_BCH), 128, 256);
        tc_mma_bf16(tbase, ad, bd, idesc, (G > 0 || kc > 0) ? 1u : 0u);
      }
      tc_commit(&bar[buf]);
    }
  }
  if (G > 0) ok = mbar_wait_bounded(&bar[(G - 1) & 1u], ((G - 1) >> 1) & 1u, NN_SPIN_LIMIT) && ok;
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  float* mine = partials + (size_t)blockIdx.x * NV;
  if (ok && warp < 4) {
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; c++) v[c] = 0.f;
    if (G > 0) tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16), v);
    // lane 32 w + lane holds row i' = d CIN + i: columns 2o + part
    const int row = 32 * warp + lane;
    if (row < NN_NDIR * CIN) {
      const int d = row / CIN, i = row - d * CIN;
#pragma unroll
      for (int o = 0; o < COUT; o++) {
        mine[((d * COUT + o) * CIN + i) * 2] = v[2 * o];
        mine[((d * COUT + o) * CIN + i) * 2 + 1] = v[2 * o + 1];
      }
    }
  } else if (!ok) {
    if (tid == 0) atomicExch(A.err, 1);
    if (G > 0) mbar_wait_bounded(&bar[(G - 1) & 1u], ((G - 1) >> 1) & 1u, NN_SPIN_LIMIT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 32);
}

// persistent grid of the tensor-core weight gradient: at most `cap` CTAs
// (the caller's partial buffer), 2 per SM (two K buffers of 108 KB each CTA)
template <int CIN, int COUT>
static cudaError_t launch_wgrad_tc(const NnLayerArgs& A, const char* delta, size_t dh,
                                   float* partials, int cap, int* grid_out, cudaStream_t st) {
  constexpr int dyn = 2 * (int)WG_BUF;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(nn_wgrad_tc_kernel<CIN, COUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nblocks = 2 * ((A.g.Vh + WG_SITES - 1) / WG_SITES);
  int grid = num_sms() * 2;
  grid = grid < nblocks ? grid : nblocks;
  grid = grid < cap ? grid : cap;
  if (grid < 1) grid = 1;
  *grid_out = grid;
  nn_wgrad_tc_kernel<CIN, COUT><<<grid, WG_THREADS, dyn, st>>>(A, delta, dh, nblocks, partials);
  return cudaGetLastError();
}

static cudaError_t nn_wgrad(int cin, int cout, const Geom& g, const void* gauge, const void* in,
                            const void* delta, float* partials, float* grad_out, int accumulate,
                            int* err, cudaStream_t st) {
  NnLayerArgs A;
  std::memset(&A, 0, sizeof(A));
  A.g = g;
  A.gauge = gauge;
  A.in = (const char*)in;
  A.in_half = nn_half_bytes(g.Vh_pad, cin);
  A.err = err;
  const size_t dh = nn_half_bytes(g.Vh_pad, cout);
  // the partial buffer holds one gradient per 128-site tile
  const int cap = 2 * ((g.Vh + NN_TILE - 1) / NN_TILE);
  int grid = 1;
  cudaError_t e;
  if (cin == 4 && cout == 8)
    e = launch_wgrad_tc<4, 8>(A, (const char*)delta, dh, partials, cap, &grid, st);
  else if (cin == 8 && cout == 8)
    e = launch_wgrad_tc<8, 8>(A, (const char*)delta, dh, partials, cap, &grid, st);
  else if (cin == 8 && cout == 4)
    e = launch_wgrad_tc<8, 4>(A, (const char*)delta, dh, partials, cap, &grid, st);
  else
    return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  const int n = NN_NDIR * cout * cin * 2;
  nn_sum_tiles<<<(n + 127) / 128, 128, 0, st>>>(partials, grid, n, grad_out, accumulate);
  return cudaGetLastError();
}

// adjoint weights: W'_e[i][o] = conj(W_{opp(e)}[o][i]); opp swaps +mu and -mu
__global__ void nn_adjoint_weights(const float* w, float* wa, int cin, int cout) {
  const int n = NN_NDIR * cout * cin;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int e = t / (cin * cout), rem = t - e * cin * cout;
    const int i = rem / cout, o = rem - i * cout;   // wa layout [e][i][o]
    const int d = e == 0 ? 0 : ((e & 1) ? e + 1 : e - 1);
    wa[t * 2] = w[((d * cout + o) * cin + i) * 2];
    wa[t * 2 + 1] = -w[((d * cout + o) * cin + i) * 2 + 1];
  }
}

// ---------------------------------------------------------------------------
// training data: complex Gaussian spinors from counter-based SplitMix64 +
// Box-Muller (the same published definitions as the host-side generator:
// draw j of stream `key` is finalise(key + (j+1) * GAMMA); complex number j
// uses uniforms 2j and 2j+1), written straight into the packed FP32 layout
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long sm64_finalise(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double sm64_uniform(unsigned long long key, unsigned long long ctr) {
  const unsigned long long z = sm64_finalise(key + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
  return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

unsigned long long sm64_stream_key(unsigned long long seed, unsigned long long stream) {
  if (stream == 0) return seed;
  unsigned long long z = (seed ^ (stream * 0xD1B54A32D192ED03ull)) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// field sample `sample` (counter offset sample * V * 12) of stream key
__global__ void gaussian_spinor_kernel(char* out, unsigned long long key, unsigned long long first,
                                       Geom g, size_t half) {
  const long long V = 2LL * g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x) {
    int x[4];
    long long r = i;
    for (int m = 0; m < 4; m++) {
      x[m] = (int)(r % g.L[m]);
      r /= g.L[m];
    }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int cb = (int)(i >> 1);
    cx<float> v[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const unsigned long long j = first + (unsigned long long)i * 12 + k;
      // FP32 transcendental functions (GB300 runs FP64 at 1/64 rate)
      const float u1 = (float)sm64_uniform(key, 2 * j), u2 = (float)sm64_uniform(key, 2 * j + 1);
      const float rad = sqrtf(-logf(u1));
      float sn, cs;
      sincosf(6.2831853071795865f * u2, &sn, &cs);
      v[k] = mk<float>(rad * cs, rad * sn);
    }
    store_spinor<WD_F32, float>(out + par * half, cb, g.Vh_pad, v);
  }
}

// Adam on the real and imaginary parts (Kingma and Ba, ICLR 2015)
__global__ void nn_adam(float* w, const float* grad, float* m, float* v, int n, float lr,
                        float b1, float b2, float eps, int step, float gscale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float gj = grad[j] * gscale;
  const float mj = b1 * m[j] + (1.f - b1) * gj;
  const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  const float mh = mj / (1.f - powf(b1, (float)step));
  const float vh = vj / (1.f - powf(b2, (float)step));
  w[j] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// network application
// ---------------------------------------------------------------------------

// the BF16 link copy of the inference layers from the packed FP32 12-real
// links (rows 0 and 1 rounded to BF16; padding sites converted as they are)
__global__ void nn_gauge_to_bf16(const float4* __restrict__ g32, int4* __restrict__ ga,
                                 int2* __restrict__ gb, int vh_pad) {
  const long n = 8L * vh_pad;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / vh_pad), cb = (int)(i - (long)r * vh_pad);
    const float4* p = g32 + (size_t)r * vh_pad * 3;
    const float4 a = __ldg(p + sbi(cb, 0, 3)), b = __ldg(p + sbi(cb, 1, 3)),
                 c = __ldg(p + sbi(cb, 2, 3));
    const __nv_bfloat162 h[6] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                                 __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w),
                                 __floats2bfloat162_rn(c.x, c.y), __floats2bfloat162_rn(c.z, c.w)};
    ga[i] = make_int4((int)bf2_u(h[0]), (int)bf2_u(h[1]), (int)bf2_u(h[2]), (int)bf2_u(h[3]));
    gb[i] = make_int2((int)bf2_u(h[4]), (int)bf2_u(h[5]));
  }
}

static cudaError_t nn_gauge_bf16(void* gbf, const void* g32, const Geom& g, cudaStream_t st) {
  int4* ga = (int4*)gbf;
  int2* gb = (int2*)((char*)gbf + (size_t)8 * g.Vh_pad * 16);
  nn_gauge_to_bf16<<<blas_grid(8LL * g.Vh_pad, 256), 256, 0, st>>>((const float4*)g32, ga, gb,
                                                                   g.Vh_pad);
  return cudaGetLastError();
}

struct NnBuffers {
  void* h1 = nullptr;  // 8 channels
  void* h2 = nullptr;  // 8 channels
  size_t bytes8 = 0;
};

static cudaError_t nn_forward(const Geom& g, const void* gauge, const float* w, const void* in,
                              void* out, NnBuffers& B, int* err, cudaStream_t st) {
  cudaError_t e;
  if ((e = nn_layer(4, 8, g, gauge, in, B.h1, w + nn_layer_offset(0), err, st))) return e;
  if ((e = nn_layer(8, 8, g, gauge, B.h1, B.h2, w + nn_layer_offset(1), err, st))) return e;
  return nn_layer(8, 4, g, gauge, B.h2, out, w + nn_layer_offset(2), err, st);
}

// One layer of the BF16 inference path: bin/bout select BF16 activations for
// the input/output (FP32 otherwise), with the parity restriction of nn_layer.
static cudaError_t nn_layer_bf16(int cin, int cout, bool bin, bool bout, const Geom& g,
                                 const void* gauge, const void* in, void* out, const float* w,
                                 int* err, cudaStream_t st, int out_parity, int zero_in) {
  NnLayerArgs A;
  A.g = g;
  A.gauge = gauge;
  A.in = (const char*)in;
  A.out = (char*)out;
  A.in_half = bin ? nn_half_bytes_bf16(g.Vh_pad, cin) : nn_half_bytes(g.Vh_pad, cin);
  A.out_half = bout ? nn_half_bytes_bf16(g.Vh_pad, cout) : nn_half_bytes(g.Vh_pad, cout);
  A.w = w;
  A.err = err;
  A.p0 = out_parity < 0 ? 0 : out_parity;
  A.np = out_parity < 0 ? 2 : 1;
  A.zero_in = zero_in;
  const int ntiles = A.np * ((g.Vh + NN_TILE - 1) / NN_TILE);
  // the one-thread-per-site kernel where the tiles fill two waves of it,
  // else the two-thread kernel (bit-identical results either way)
  cudaError_t e = cudaErrorNotReady;
  if (WD_NN_INFER1) {
    if (cin == 4 && cout == 8 && !bin && bout) e = launch_infer<4, 8, false, true>(A, ntiles, st);
    if (cin == 8 && cout == 8 && bin && bout) e = launch_infer<8, 8, true, true>(A, ntiles, st);
    if (cin == 8 && cout == 4 && bin && !bout) e = launch_infer<8, 4, true, false>(A, ntiles, st);
  }
  if (e != cudaErrorNotReady) return e;
  if (cin == 4 && cout == 8 && !bin && bout) return launch_layer<4, 8, false, true>(A, ntiles, st);
  if (cin == 8 && cout == 8 && bin && bout) return launch_layer<8, 8, true, true>(A, ntiles, st);
  if (cin == 8 && cout == 4 && bin && !bout) return launch_layer<8, 4, true, false>(A, ntiles, st);
  return cudaErrorInvalidValue;
}

// N (even: P_e N P_e) with BF16 activations between the layers (input and output stay
// packed FP32 fields; gauge: the BF16 link copy, nn_gauge_bf16): the link
// transport runs in packed bf16x2 arithmetic,
// the channel mixing on the tensor cores with FP32 accumulation.  For the
// preconditioner inside the flexible CG, whose beta absorbs the extra
// rounding (about 2^-8 relative per layer).  B.h1 and B.h2 hold 8-channel
// BF16 fields here.
static cudaError_t nn_forward_bf16(const Geom& g, const void* gauge, const float* w,
                                   const void* in, void* out, NnBuffers& B, int* err,
                                   cudaStream_t st, bool even) {
  cudaError_t e;
  if ((e = nn_layer_bf16(4, 8, false, true, g, gauge, in, B.h1, w + nn_layer_offset(0), err, st,
                         -1, even ? WD_ODD : -1)))
    return e;
  if ((e = nn_layer_bf16(8, 8, true, true, g, gauge, B.h1, B.h2, w + nn_layer_offset(1), err, st,
                         -1, -1)))
    return e;
  return nn_layer_bf16(8, 4, true, false, g, gauge, B.h2, out, w + nn_layer_offset(2), err, st,
                       even ? WD_EVEN : -1, -1);
}

// The even-even block P_e N P_e: the odd half of `in` is taken as zero and
// never read (the first layer's even sites keep only their self term, its
// odd sites only their hops), and the last layer computes the even sites
// only (the odd half of `out` is left as it was).  About 2/3 of the work of
// the full network.
static cudaError_t nn_forward_even(const Geom& g, const void* gauge, const float* w,
                                   const void* in, void* out, NnBuffers& B, int* err,
                                   cudaStream_t st) {
  cudaError_t e;
  if ((e = nn_layer(4, 8, g, gauge, in, B.h1, w + nn_layer_offset(0), err, st, -1, WD_ODD)))
    return e;
  if ((e = nn_layer(8, 8, g, gauge, B.h1, B.h2, w + nn_layer_offset(1), err, st))) return e;
  return nn_layer(8, 4, g, gauge, B.h2, out, w + nn_layer_offset(2), err, st, WD_EVEN);
}

// (1 + c kappa H) on the first four channels of a layer; identity on the rest
static void init_hopping_layer(float* w, int cin, int cout, double cr, double ci, double kappa) {
  // chiral basis: gamma_mu = [[0, A_mu], [A_mu^+, 0]], A = -i sigma_{1,2,3}, A_t = 1
  const double SX[2][2][2] = {{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}};
  const double SY[2][2][2] = {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}};
  const double SZ[2][2][2] = {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}};
  double gam[4][4][4][2];
  std::memset(gam, 0, sizeof(gam));
  const double(*S[3])[2][2] = {SX, SY, SZ};
  for (int mu = 0; mu < 4; mu++)
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        double re, im;  // A_mu[a][b]
        if (mu < 3) {   // -i sigma
          re = S[mu][a][b][1];
          im = -S[mu][a][b][0];
        } else {
          re = a == b ? 1.0 : 0.0;
          im = 0.0;
        }
        gam[mu][a][b + 2][0] = re;       // upper right: A
        gam[mu][a][b + 2][1] = im;
        gam[mu][b + 2][a][0] = re;       // lower left: A^+ (conjugate transpose)
        gam[mu][b + 2][a][1] = -im;
      }
  std::memset(w, 0, sizeof(float) * 9 * cout * cin * 2);
  auto W = [&](int d, int o, int i) -> float* { return w + ((d * cout + o) * cin + i) * 2; };
  for (int o = 0; o < cout && o < cin; o++) W(0, o, o)[0] = 1.f;
  for (int mu = 0; mu < 4; mu++)
    for (int fb = 0; fb < 2; fb++) {
      const int d = 1 + 2 * mu + fb;
      const double sgn = fb == 0 ? -1.0 : 1.0;  // (1 - gamma) forward, (1 + gamma) backward
      for (int o = 0; o < 4; o++)
        for (int i = 0; i < 4; i++) {
          double pr = (o == i ? 1.0 : 0.0) + sgn * gam[mu][o][i][0];
          double pi = sgn * gam[mu][o][i][1];
          // times c kappa
          const double vr = kappa * (cr * pr - ci * pi), vi = kappa * (cr * pi + ci * pr);
          W(d, o, i)[0] = (float)vr;
          W(d, o, i)[1] = (float)vi;
        }
    }
}

void nn_init_hopping_series(float* w_host, double kappa) {
  // (1 + k H)(1 + i k H)(1 - i k H) = 1 + kH + k^2 H^2 + k^3 H^3
  init_hopping_layer(w_host + nn_layer_offset(0), 4, 8, 1.0, 0.0, kappa);
  init_hopping_layer(w_host + nn_layer_offset(1), 8, 8, 0.0, 1.0, kappa);
  init_hopping_layer(w_host + nn_layer_offset(2), 8, 4, 0.0, -1.0, kappa);
}


// ---------------------------------------------------------------------------
// flexible GCR kernels (classical Gram-Schmidt in one pass each)
// ---------------------------------------------------------------------------

constexpr int GCR_MAXK = 16;

struct PtrList {
  const char* p[GCR_MAXK];
};

// res[j] = <v_j, w> (complex), j < k; packed FP32 full fields
__global__ void __launch_bounds__(256) multi_cdot_kernel(const PtrList vs, int k, const char* w,
                                                         Geom g, size_t half, RedScratch rs,
                                                         double* res) {
  float acc[2 * GCR_MAXK];
#pragma unroll
  for (int j = 0; j < 2 * GCR_MAXK; j++) acc[j] = 0.f;
  const long long n = 2LL * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> a[12];
    load_spinor_rw<WD_F32, float>(a, w + h * half, cb, g.Vh_pad);
#pragma unroll
    for (int j = 0; j < GCR_MAXK; j++) {
      if (j < k) {
        cx<float> b[12];
        load_spinor_rw<WD_F32, float>(b, vs.p[j] + h * half, cb, g.Vh_pad);
        site_cdot(b, a, acc[2 * j], acc[2 * j + 1]);
      }
    }
  }
  double tot[2 * GCR_MAXK];
  if (grid_reduce<2 * GCR_MAXK, 256>(acc, rs, tot) && threadIdx.x == 0) {
    for (int j = 0; j < 2 * k; j++) res[j] = tot[j];
  }
}

// w -= sum_j beta_j W_j ; z -= sum_j beta_j Z_j ; beta_j = dots[j] / nrm[j]
__global__ void __launch_bounds__(256) multi_axpy_kernel(const PtrList Ws, const PtrList Zs, int k,
                                                         char* w, char* z, const double* dots,
                                                         const double* nrm, Geom g, size_t half) {
  float br[GCR_MAXK], bi[GCR_MAXK];
#pragma unroll
  for (int j = 0; j < GCR_MAXK; j++) {
    br[j] = j < k ? (float)(dots[2 * j] / nrm[j]) : 0.f;
    bi[j] = j < k ? (float)(dots[2 * j + 1] / nrm[j]) : 0.f;
  }
  const long long n = 2LL * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> a[12], c[12];
    load_spinor_rw<WD_F32, float>(a, w + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(c, z + h * half, cb, g.Vh_pad);
#pragma unroll
    for (int j = 0; j < GCR_MAXK; j++) {
      if (j < k) {
        cx<float> u[12], v[12];
        load_spinor_rw<WD_F32, float>(u, Ws.p[j] + h * half, cb, g.Vh_pad);
        load_spinor_rw<WD_F32, float>(v, Zs.p[j] + h * half, cb, g.Vh_pad);
#pragma unroll
        for (int q = 0; q < 12; q++) {
          a[q].r -= br[j] * u[q].r - bi[j] * u[q].i;
          a[q].i -= br[j] * u[q].i + bi[j] * u[q].r;
          c[q].r -= br[j] * v[q].r - bi[j] * v[q].i;
          c[q].i -= br[j] * v[q].i + bi[j] * v[q].r;
        }
      }
    }
    store_spinor<WD_F32, float>(w + h * half, cb, g.Vh_pad, a);
    store_spinor<WD_F32, float>(z + h * half, cb, g.Vh_pad, c);
  }
}

// out[0] = ||w||^2, out[1..2] = <w, r>
__global__ void __launch_bounds__(256) norm_cdot_kernel(const char* w, const char* r, Geom g,
                                                        size_t half, RedScratch rs, double* out) {
  float acc[3] = {0.f, 0.f, 0.f};
  const long long n = 2LL * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> a[12], b[12];
    load_spinor_rw<WD_F32, float>(a, w + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(b, r + h * half, cb, g.Vh_pad);
    acc[0] += site_norm2<float>(a);
    site_cdot(a, b, acc[1], acc[2]);
  }
  double tot[3];
  if (grid_reduce<3, 256>(acc, rs, tot) && threadIdx.x == 0) {
    out[0] = tot[0];
    out[1] = tot[1];
    out[2] = tot[2];
  }
}

// x += alpha z ; r -= alpha w ; out = ||r||^2 ; alpha = wr / ww
__global__ void __launch_bounds__(256) gcr_update_kernel(char* x, char* r, const char* z,
                                                         const char* w, const double* nc, Geom g,
                                                         size_t half, RedScratch rs, double* out) {
  const float ar = (float)(nc[1] / nc[0]), ai = (float)(nc[2] / nc[0]);
  float acc[1] = {0.f};
  const long long n = 2LL * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> xv[12], rv[12], zv[12], wv[12];
    load_spinor_rw<WD_F32, float>(xv, x + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(rv, r + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(zv, z + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(wv, w + h * half, cb, g.Vh_pad);
#pragma unroll
    for (int q = 0; q < 12; q++) {
      xv[q].r += ar * zv[q].r - ai * zv[q].i;
      xv[q].i += ar * zv[q].i + ai * zv[q].r;
      rv[q].r -= ar * wv[q].r - ai * wv[q].i;
      rv[q].i -= ar * wv[q].i + ai * wv[q].r;
    }
    store_spinor<WD_F32, float>(x + h * half, cb, g.Vh_pad, xv);
    store_spinor<WD_F32, float>(r + h * half, cb, g.Vh_pad, rv);
    acc[0] += site_norm2<float>(rv);
  }
  double tot[1];
  if (grid_reduce<1, 256>(acc, rs, tot) && threadIdx.x == 0) out[0] = tot[0];
}

// x64 += xs (F32 -> F64; nh halves: 2 full fields, 1 the even sites); xs = 0
__global__ void accumulate_full_kernel(char* x64, char* xs, Geom g, size_t h64, size_t h32,
                                       int nh = 2) {
  const long long n = (long long)nh * g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<double> a[12];
    cx<float> b[12];
    load_spinor_rw<WD_F64, double>(a, x64 + h * h64, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(b, xs + h * h32, cb, g.Vh_pad);
#pragma unroll
    for (int q = 0; q < 12; q++) {
      a[q].r += (double)b[q].r;
      a[q].i += (double)b[q].i;
      b[q] = mk<float>(0.f, 0.f);
    }
    store_spinor<WD_F64, double>(x64 + h * h64, cb, g.Vh_pad, a);
    store_spinor<WD_F32, float>(xs + h * h32, cb, g.Vh_pad, b);
  }
}


// ---------------------------------------------------------------------------
// flexible CG on normal equations A^+ A x = A^+ b with the preconditioner
// N N^+ (N the network): packed FP32 fields of nh halves (nh = 1: the even
// sites), scalars on the device.
// rho[kp] = <s, z> of the current iteration, rho[1-kp] that of the next one;
// qq[0..1] = ||D p||^2 on the even / odd half.
// ---------------------------------------------------------------------------

struct FcgScalars {
  double rho[2];
  double zeta;    // <s_old, z_new>: the Polak-Ribiere correction of beta
  double qq[2];
  double rr;      // ||r||^2, r = b - D x (sloppy)
  double r64;     // ||b - D x64||^2 (FP64)
  double bn;      // ||b||^2
};

// x += alpha p ; r -= alpha q ; rr = ||r||^2 ; alpha = rho[kp] / ||q||^2
__global__ void __launch_bounds__(256) fcg_update_xr(char* x, char* r, const char* p,
                                                     const char* q, FcgScalars* sc, int kp,
                                                     Geom g, size_t half, int nh, RedScratch rs) {
  const float a = (float)(sc->rho[kp] / (sc->qq[0] + sc->qq[1]));
  float acc[1] = {0.f};
  const long long n = (long long)nh * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> xv[12], rv[12], pv[12], qv[12];
    load_spinor_rw<WD_F32, float>(xv, x + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(rv, r + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(pv, p + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(qv, q + h * half, cb, g.Vh_pad);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      xv[k].r = fmaf(a, pv[k].r, xv[k].r);
      xv[k].i = fmaf(a, pv[k].i, xv[k].i);
      rv[k].r = fmaf(-a, qv[k].r, rv[k].r);
      rv[k].i = fmaf(-a, qv[k].i, rv[k].i);
    }
    store_spinor<WD_F32, float>(x + h * half, cb, g.Vh_pad, xv);
    store_spinor<WD_F32, float>(r + h * half, cb, g.Vh_pad, rv);
    acc[0] += site_norm2<float>(rv);
  }
  double tot[1];
  if (grid_reduce<1, 256>(acc, rs, tot) && threadIdx.x == 0) sc->rr = tot[0];
}

// rho[slot] = Re <s, z> ; zeta = Re <s_old, z> (s_old may be null: zeta = 0)
__global__ void __launch_bounds__(256) fcg_dots(const char* s, const char* s_old, const char* z,
                                                FcgScalars* sc, int slot, Geom g, size_t half,
                                                int nh, RedScratch rs) {
  float acc[3] = {0.f, 0.f, 0.f};
  const long long n = (long long)nh * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> sv[12], zv[12];
    load_spinor_rw<WD_F32, float>(sv, s + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(zv, z + h * half, cb, g.Vh_pad);
    site_cdot(sv, zv, acc[0], acc[1]);
    if (s_old) {
      load_spinor_rw<WD_F32, float>(sv, s_old + h * half, cb, g.Vh_pad);
      float im = 0.f;
      site_cdot(sv, zv, acc[2], im);
    }
  }
  double tot[3];
  if (grid_reduce<3, 256>(acc, rs, tot) && threadIdx.x == 0) {
    sc->rho[slot] = tot[0];
    sc->zeta = tot[2];
  }
}

// p = z + beta p, beta = (rho[1-kp] - zeta) / rho[kp]  (restart: p = z)
__global__ void __launch_bounds__(256) fcg_update_p(char* p, const char* z, const FcgScalars* sc,
                                                    int kp, int restart, Geom g, size_t half,
                                                    int nh) {
  const float beta = restart ? 0.f : (float)((sc->rho[1 - kp] - sc->zeta) / sc->rho[kp]);
  const long long n = (long long)nh * g.Vh;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int h = (int)(i / g.Vh), cb = (int)(i - (long long)h * g.Vh);
    cx<float> pv[12], zv[12];
    load_spinor_rw<WD_F32, float>(pv, p + h * half, cb, g.Vh_pad);
    load_spinor_rw<WD_F32, float>(zv, z + h * half, cb, g.Vh_pad);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      pv[k].r = restart ? zv[k].r : fmaf(beta, pv[k].r, zv[k].r);
      pv[k].i = restart ? zv[k].i : fmaf(beta, pv[k].i, zv[k].i);
    }
    store_spinor<WD_F32, float>(p + h * half, cb, g.Vh_pad, pv);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct Alloc {
  std::vector<void*> ptrs;
  cudaError_t get(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Alloc() {
    for (void* p : ptrs) cudaFree(p);
  }
};

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// out = in - kappa H in on packed full fields (a = -kappa) or the variant
// out = in - D in ... through the single-field kernel
cudaError_t full_op(int prec, int recon, const void* gauge, void* out, const void* in,
                    double kappa, const Geom& g, cudaStream_t st, const void* bfield = nullptr,
                    bool dagger = false) {
  const size_t h = spinor_half_bytes(g, prec);
  for (int p = 0; p < 2; p++) {
    DslashArgs d;
    d.out = (char*)out + p * h;
    d.in = (const char*)in + (1 - p) * h;
    d.gauge = gauge;
    if (bfield) {
      // out = b - D in = b - in + kappa H in
      d.a = kappa;
      d.x = (const char*)bfield + p * h;
      d.bx = 1.0;
      d.y = (const char*)in + p * h;
      d.cy = -1.0;
    } else {
      d.a = -kappa;
      d.x = (const char*)in + p * h;
      d.bx = 1.0;
      d.y = nullptr;
      d.cy = 0.0;
    }
    d.norm_out = nullptr;
    d.rs = scratch();
    d.g = g;
    d.parity = p;
    cudaError_t e = launch_dslash(prec, d, recon, dagger, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

#define NCK(call)                                 \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      state().last_cuda_error = (int)e_;          \
      return WD_ERR_CUDA;                         \
    }                                             \
  } while (0)

}  // namespace

int nn_apply_impl(void* out, const void* in, const float* w, const void* gauge, const int dims[4]) {
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  Alloc al;
  NnBuffers B;
  B.bytes8 = 2 * nn_half_bytes(g.Vh_pad, 8);
  NCK(al.get(&B.h1, B.bytes8));
  NCK(al.get(&B.h2, B.bytes8));
  int* flag = nullptr;
  NCK(device_flag(&flag, st));
  NCK(nn_forward(g, gauge, w, in, out, B, flag, st));
  int hflag = 0;
  NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  return hflag ? WD_ERR_TIMEOUT : WD_OK;
}

// out = N(in) (flags & 2: only the even-even block P_e N P_e, the odd half of
// in taken as zero and the odd half of out untouched), with FP32 (flags & 1
// == 0) or BF16 activations between the layers
int nn_apply_ex_impl(void* out, const void* in, const float* w, const void* gauge,
                     const int dims[4], int flags) {
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  Alloc al;
  NnBuffers B;
  B.bytes8 = 2 * nn_half_bytes(g.Vh_pad, 8);
  NCK(al.get(&B.h1, B.bytes8));
  NCK(al.get(&B.h2, B.bytes8));
  int* flag = nullptr;
  NCK(device_flag(&flag, st));
  const bool even = (flags & 2) != 0;
  if (flags & 1) {
    void* gbf;
    NCK(al.get(&gbf, nn_gauge_bytes_bf16(g.Vh_pad)));
    NCK(nn_gauge_bf16(gbf, gauge, g, st));
    NCK(nn_forward_bf16(g, gbf, w, in, out, B, flag, st, even));
  }
  else if (even)
    NCK(nn_forward_even(g, gauge, w, in, out, B, flag, st));
  else
    NCK(nn_forward(g, gauge, w, in, out, B, flag, st));
  int hflag = 0;
  NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  return hflag ? WD_ERR_TIMEOUT : WD_OK;
}

int nn_layer_impl(void* out, const void* in, const float* w, int cin, int cout, const void* gauge,
                  const int dims[4]) {
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  int* flag = nullptr;
  NCK(device_flag(&flag, st));
  NCK(nn_layer(cin, cout, g, gauge, in, out, w, flag, st));
  int hflag = 0;
  NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  return hflag ? WD_ERR_TIMEOUT : WD_OK;
}

int nn_wgrad_impl(float* grad, const void* in, const void* delta, int cin, int cout,
                  const void* gauge, const int dims[4]) {
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  Alloc al;
  void* part;
  const int ntile = 2 * ((g.Vh + NN_TILE - 1) / NN_TILE);
  NCK(al.get(&part, (size_t)ntile * NN_NDIR * cout * cin * 2 * sizeof(float)));
  int* flag = nullptr;
  NCK(device_flag(&flag, st));
  NCK(nn_wgrad(cin, cout, g, gauge, in, delta, (float*)part, grad, 0, flag, st));
  int hflag = 0;
  NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  return hflag ? WD_ERR_TIMEOUT : WD_OK;
}

int gaussian_spinor_impl(void* out, unsigned long long seed, unsigned long long stream,
                         unsigned long long first, const int dims[4]) {
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  gaussian_spinor_kernel<<<blas_grid(2LL * g.Vh, 256), 256, 0, st>>>(
      (char*)out, sm64_stream_key(seed, stream), first, g, spinor_half_bytes(g, WD_F32));
  NCK(cudaGetLastError());
  return WD_OK;
}

int nn_init_impl(float* w_dev, double kappa) {
  std::vector<float> h(NN_PARAMS);
  nn_init_hopping_series(h.data(), kappa);
  NCK(cudaMemcpy(w_dev, h.data(), NN_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
  return WD_OK;
}

int nn_train_impl(float* w, const double* gauge, double kappa, const int dims[4],
                  const wd_nn_train_params* prm, wd_nn_train_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  wd_nn_train_params P = *prm;
  if (P.samples < 1 || P.batch < 1 || P.epochs < 1 || !(P.lr > 0) || P.smooth < 0)
    return WD_ERR_ARG;
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  Alloc al;
  const size_t V = 2 * (size_t)g.Vh;
  const size_t h32 = spinor_half_bytes(g, WD_F32);
  // packed FP32 links (network transport and the operator that draws b)
  void* gp;
  NCK(al.get(&gp, gauge_bytes(g, WD_F32, 12)));
  const double* gd = gauge;
  if (!on_device(gauge)) {
    void* v;
    NCK(al.get(&v, 4 * V * 18 * sizeof(double)));
    NCK(cudaMemcpyAsync(v, gauge, 4 * V * 18 * sizeof(double), cudaMemcpyHostToDevice, st));
    gd = (const double*)v;
  }
  NCK(pack_gauge(gp, gd, g, WD_F32, 12, st));
  if (P.init) NCK((cudaError_t)(nn_init_impl(w, kappa) == WD_OK ? cudaSuccess : cudaErrorUnknown));
  void *x, *b, *y, *dl, *wa, *grad, *m, *v2, *part, *losses;
  NnBuffers B;
  B.bytes8 = 2 * nn_half_bytes(g.Vh_pad, 8);
  void *d1, *d2;
  NCK(al.get(&x, 2 * h32));
  NCK(al.get(&b, 2 * h32));
  NCK(al.get(&y, 2 * h32));
  NCK(al.get(&dl, 2 * h32));
  NCK(al.get(&B.h1, B.bytes8));
  NCK(al.get(&B.h2, B.bytes8));
  NCK(al.get(&d1, B.bytes8));
  NCK(al.get(&d2, B.bytes8));
  NCK(al.get(&wa, NN_PARAMS * sizeof(float)));
  NCK(al.get(&grad, NN_PARAMS * sizeof(float)));
  NCK(al.get(&m, NN_PARAMS * sizeof(float)));
  NCK(al.get(&v2, NN_PARAMS * sizeof(float)));
  const int ntile = 2 * ((g.Vh + NN_TILE - 1) / NN_TILE);
  NCK(al.get(&part, (size_t)ntile * NN_NDIR * 8 * 8 * 2 * sizeof(float)));
  const int steps_per_epoch = (P.samples + P.batch - 1) / P.batch;
  const int nsteps = steps_per_epoch * P.epochs;
  NCK(al.get(&losses, (size_t)nsteps * 2 * sizeof(double)));
  NCK(cudaMemsetAsync(m, 0, NN_PARAMS * sizeof(float), st));
  NCK(cudaMemsetAsync(v2, 0, NN_PARAMS * sizeof(float), st));
  NCK(cudaMemsetAsync(losses, 0, (size_t)nsteps * 2 * sizeof(double), st));
  int* flag = nullptr;
  NCK(device_flag(&flag, st));
  NCK(ensure_scratch(4096));
  const unsigned long long key = sm64_stream_key(P.seed, 7);
  float* W = w;
  float* WA = (float*)wa;
  const int grid = blas_grid(V, 256);
  for (int step = 0; step < nsteps; step++) {
    // adjoint weights of layers 2 and 3 (for the input gradients)
    nn_adjoint_weights<<<8, 256, 0, st>>>(W + nn_layer_offset(1), WA + nn_layer_offset(1), 8, 8);
    nn_adjoint_weights<<<8, 256, 0, st>>>(W + nn_layer_offset(2), WA + nn_layer_offset(2), 8, 4);
    NCK(cudaGetLastError());
    for (int sbt = 0; sbt < P.batch; sbt++) {
      const long long sample = ((long long)step * P.batch + sbt) % P.samples;
      gaussian_spinor_kernel<<<grid, 256, 0, st>>>((char*)x, key,
                                                   (unsigned long long)sample * V * 12, g, h32);
      NCK(cudaGetLastError());
      if (P.smooth > 0 && (sample & 1)) {
        // x <- x - w D^+ D x damps the large singular values of D (y and dl
        // are free at this point and serve as the two temporaries)
        const double wd = 1.0 / ((1.0 + 8.0 * kappa) * (1.0 + 8.0 * kappa));
        for (int k = 0; k < P.smooth; k++) {
          NCK(full_op(WD_F32, 12, gp, y, x, kappa, g, st));
          NCK(full_op(WD_F32, 12, gp, dl, y, kappa, g, st, nullptr, true));
          NCK(axpby(-wd, dl, 1.0, x, g, WD_F32, 2, st));
        }
      }
      NCK(full_op(WD_F32, 12, gp, b, x, kappa, g, st));                    // b = D x
      NCK(nn_forward(g, gp, W, b, y, B, flag, st));                        // y = N(b)
      NCK(axpby(1.0, y, 0.0, dl, g, WD_F32, 2, st));                       // dl = y
      NCK(axpby(-1.0, x, 1.0, dl, g, WD_F32, 2, st));                      // dl = y - x
      // the loss of the batch's last sample: ||y - x||^2 and ||x||^2
      double* L = (double*)losses + 2 * step;
      NCK(norm2(L + 0, dl, g, WD_F32, 2, st));
      NCK(norm2(L + 1, x, g, WD_F32, 2, st));
      // backward: G3 (h2 -> y), delta2 = L3^+ dl, G2, delta1 = L2^+ delta2, G1
      const int acc = sbt > 0;
      NCK(nn_wgrad(8, 4, g, gp, B.h2, dl, (float*)part, (float*)grad + nn_layer_offset(2), acc,
                   flag, st));
      NCK(nn_layer(4, 8, g, gp, dl, d2, WA + nn_layer_offset(2), flag, st));
      NCK(nn_wgrad(8, 8, g, gp, B.h1, d2, (float*)part, (float*)grad + nn_layer_offset(1), acc,
                   flag, st));
      NCK(nn_layer(8, 8, g, gp, d2, d1, WA + nn_layer_offset(1), flag, st));
      NCK(nn_wgrad(4, 8, g, gp, b, d1, (float*)part, (float*)grad + nn_layer_offset(0), acc,
                   flag, st));
    }
    const float gscale = (float)(1.0 / ((double)P.batch * 12.0 * (double)V));
    nn_adam<<<(NN_PARAMS + 255) / 256, 256, 0, st>>>(W, (const float*)grad, (float*)m, (float*)v2,
                                                    NN_PARAMS, P.lr, 0.9f, 0.999f, 1e-8f, step + 1,
                                                    gscale);
    NCK(cudaGetLastError());
  }
  std::vector<double> hl((size_t)nsteps * 2);
  NCK(cudaMemcpyAsync(hl.data(), losses, hl.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  int hflag = 0;
  NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->steps = nsteps;
    info->loss_first = hl[1] > 0 ? hl[0] / hl[1] : 0.0;
    info->loss_last = hl[2 * nsteps - 1] > 0 ? hl[2 * nsteps - 2] / hl[2 * nsteps - 1] : 0.0;
    info->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return hflag ? WD_ERR_TIMEOUT : WD_OK;
}

// flexible GCR(m) on the full operator D, preconditioned by the network
// (w == nullptr: no preconditioner), FP32 inner vectors, FP64 restarts
int fgcr_impl(double* x, const double* bsrc, const double* gauge, double kappa,
              const int dims[4], const float* wts, const wd_solve_params* prm,
              wd_solve_info* info, int m) {
  const auto t0 = std::chrono::steady_clock::now();
  wd_solve_params P;
  wd_solve_params_default(&P);
  if (prm) P = *prm;
  if (m < 1 || m > GCR_MAXK) return WD_ERR_ARG;
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  Alloc al;
  const size_t V = 2 * (size_t)g.Vh;
  const size_t h32 = spinor_half_bytes(g, WD_F32), h64 = spinor_half_bytes(g, WD_F64);
  void *g32, *g64;
  NCK(al.get(&g32, gauge_bytes(g, WD_F32, 12)));
  NCK(al.get(&g64, gauge_bytes(g, WD_F64, 18)));
  const double* gd = gauge;
  if (!on_device(gauge)) {
    void* v;
    NCK(al.get(&v, 4 * V * 18 * sizeof(double)));
    NCK(cudaMemcpyAsync(v, gauge, 4 * V * 18 * sizeof(double), cudaMemcpyHostToDevice, st));
    gd = (const double*)v;
  }
  NCK(pack_gauge(g32, gd, g, WD_F32, 12, st));
  NCK(pack_gauge(g64, gd, g, WD_F64, 18, st));
  const double* bd = bsrc;
  double* canon = nullptr;
  {
    void* v;
    NCK(al.get(&v, V * 24 * sizeof(double)));
    canon = (double*)v;
  }
  if (!on_device(bsrc)) {
    NCK(cudaMemcpyAsync(canon, bsrc, V * 24 * sizeof(double), cudaMemcpyHostToDevice, st));
    bd = canon;
  }
  void *b64, *x64, *r64, *r, *xs, *zs, *ws, *scal;
  NCK(al.get(&b64, 2 * h64));
  NCK(al.get(&x64, 2 * h64));
  NCK(al.get(&r64, 2 * h64));
  NCK(al.get(&r, 2 * h32));
  NCK(al.get(&xs, 2 * h32));
  NCK(al.get(&zs, (size_t)m * 2 * h32));
  NCK(al.get(&ws, (size_t)m * 2 * h32));
  NCK(al.get(&scal, (size_t)(4 * GCR_MAXK + 16) * sizeof(double)));
  double* S = (double*)scal;
  double* dots = S;                       // 2 * GCR_MAXK
  double* nrm = S + 2 * GCR_MAXK;          // GCR_MAXK
  double* nc = S + 3 * GCR_MAXK;           // 3
  double* rr = nc + 3;                     // 1
  double* r64n = rr + 1;                   // 1
  double* bn = r64n + 1;                   // 1
  constexpr int I_RR = 3 * GCR_MAXK + 3, I_R64 = 3 * GCR_MAXK + 4, I_BN = 3 * GCR_MAXK + 5;
  NnBuffers B;
  B.bytes8 = 2 * nn_half_bytes(g.Vh_pad, 8);
  if (wts) {
    NCK(al.get(&B.h1, B.bytes8));
    NCK(al.get(&B.h2, B.bytes8));
  }
  int* flag = nullptr;
  NCK(device_flag(&flag, st));
  NCK(ensure_scratch((size_t)num_sms() * 8 * 2 * GCR_MAXK + 1024));
  NCK(pack_spinor(b64, bd, g, WD_FULL, WD_F64, st));
  NCK(norm2(bn, b64, g, WD_F64, 2, st));
  NCK(cudaMemsetAsync(x64, 0, 2 * h64, st));
  NCK(cudaMemsetAsync(xs, 0, 2 * h32, st));
  const int grid = blas_grid(V, 256);
  RedScratch rs = scratch();
  double hs[4 * GCR_MAXK + 16];
  auto rd = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hs, S, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
  };
  // r64 = b - D x64 ; r = r64
  auto restart = [&]() -> cudaError_t {
    cudaError_t e = full_op(WD_F64, 18, g64, r64, x64, kappa, g, st, b64);
    if (e == cudaSuccess) e = norm2(r64n, r64, g, WD_F64, 2, st);
    if (e == cudaSuccess) e = convert_spinor(r, WD_F32, r64, WD_F64, g, 2, st);
    return e;
  };
  NCK(restart());
  NCK(rd());
  const double bnorm = std::sqrt(hs[I_BN]);
  const double target = P.tol * bnorm * 0.9;
  int iters = 0, status = WD_ERR_NOCONV, restarts = 0;
  double rel = bnorm > 0 ? std::sqrt(hs[I_R64]) / bnorm : 0.0;
  bool done = !(bnorm > 0) || std::sqrt(hs[I_R64]) <= target;
  while (!done && iters < P.maxiter) {
    int k = 0;
    for (; k < m && iters < P.maxiter; k++, iters++) {
      char* zk = (char*)zs + (size_t)k * 2 * h32;
      char* wk = (char*)ws + (size_t)k * 2 * h32;
      if (wts)
        NCK(nn_forward(g, g32, wts, r, zk, B, flag, st));
      else
        NCK(convert_spinor(zk, WD_F32, r, WD_F32, g, 2, st));
      NCK(full_op(WD_F32, 12, g32, wk, zk, kappa, g, st));
      if (k > 0) {
        PtrList Wl, Zl;
        for (int j = 0; j < GCR_MAXK; j++) {
          Wl.p[j] = (const char*)ws + (size_t)(j < k ? j : 0) * 2 * h32;
          Zl.p[j] = (const char*)zs + (size_t)(j < k ? j : 0) * 2 * h32;
        }
        multi_cdot_kernel<<<grid, 256, 0, st>>>(Wl, k, wk, g, h32, rs, dots);
        NCK(cudaGetLastError());
        multi_axpy_kernel<<<grid, 256, 0, st>>>(Wl, Zl, k, wk, zk, dots, nrm, g, h32);
        NCK(cudaGetLastError());
      }
      norm_cdot_kernel<<<grid, 256, 0, st>>>(wk, (const char*)r, g, h32, rs, nc);
      NCK(cudaGetLastError());
      NCK(cudaMemcpyAsync(nrm + k, nc, sizeof(double), cudaMemcpyDeviceToDevice, st));
      gcr_update_kernel<<<grid, 256, 0, st>>>((char*)xs, (char*)r, zk, wk, nc, g, h32, rs, rr);
      NCK(cudaGetLastError());
      NCK(rd());
      const double rn = std::sqrt(hs[I_RR]);
      if (!std::isfinite(rn)) {
        status = WD_ERR_NONFINITE;
        done = true;
        break;
      }
      if (rn <= target) {
        k++;
        iters++;
        break;
      }
    }
    if (status == WD_ERR_NONFINITE) break;
    accumulate_full_kernel<<<grid, 256, 0, st>>>((char*)x64, (char*)xs, g, h64, h32);
    NCK(cudaGetLastError());
    NCK(restart());
    NCK(rd());
    restarts++;
    const double r64v = std::sqrt(hs[I_R64]);
    rel = r64v / bnorm;
    if (!std::isfinite(r64v)) {
      status = WD_ERR_NONFINITE;
      break;
    }
    if (r64v <= target) done = true;
  }
  if (done && status != WD_ERR_NONFINITE) status = WD_OK;
  // unpack
  const bool xdev = on_device(x);
  double* xd = xdev ? x : canon;
  NCK(unpack_spinor(xd, x64, g, WD_FULL, WD_F64, st));
  if (!xdev) NCK(cudaMemcpyAsync(x, xd, V * 24 * sizeof(double), cudaMemcpyDeviceToHost, st));
  int hflag = 0;
  NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  if (hflag) status = WD_ERR_TIMEOUT;
  if (status == WD_OK && !(rel <= P.tol)) status = WD_ERR_NOCONV;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = iters;
    info->reliable_updates = restarts;
    info->status = status;
    info->true_residual = rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

int solve_impl(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
               const wd_solve_params* prm, wd_solve_info* info);

// Flexible CG on the even-odd preconditioned system, preconditioned by the
// network.  The even-even block of D^-1 is exactly the inverse of the Schur
// complement Mhat = 1 - kappa^2 H_eo H_oe, so the even-even block of a
// network trained as an approximate inverse of D, N_e = P_e N P_e, is an
// approximate inverse of Mhat.  CG runs on Mhat^+ Mhat x_e = Mhat^+ bhat_e
// (bhat_e = b_e + kappa H_eo b_o) with the preconditioner N_e N_e^+, which is
// Hermitian and positive definite, so CG converges whatever the spectrum of
// D; then x_o = b_o + kappa H_oe x_e.  An even-only input lets the network
// skip a third of its work (nn_forward_even).  BF16 rounding makes N_e vary
// slightly between applications; the Polak-Ribiere form of beta,
// <z_new, s_new - s_old> / <z_old, s_old> (flexible CG, Notay, SIAM J. Sci.
// Comput. 22, 2000) absorbs that.  FP32 vectors and operator, FP64 reliable
// updates (x accumulated and r = bhat - Mhat x recomputed in FP64 every
// `reliable_interval` iterations and whenever the FP32 residual looks
// converged; the search direction restarts there).  The true residual
// ||b - D x|| is computed in FP64 on the full lattice.  If this does not
// reach the tolerance (maxiter, a non-finite residual, a network wait that
// timed out), the plain mixed-precision even-odd CG continues from the best
// iterate.  wts == nullptr: CGNR on the even-odd system, no network.
int solve_impl(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
               const wd_solve_params* prm, wd_solve_info* info);

// the preconditioner of the flexible CG runs the network with BF16
// activations (1) or FP32 ones (0)
#ifndef WD_NN_FCG_BF16
#define WD_NN_FCG_BF16 1
#endif

int fcg_impl(double* x, const double* bsrc, const double* gauge, double kappa, const int dims[4],
             const float* wts, const wd_solve_params* prm, wd_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  wd_solve_params P;
  wd_solve_params_default(&P);
  if (prm) P = *prm;
  if (P.reliable_interval < 1 || P.maxiter < 1) return WD_ERR_ARG;
  const Geom g = make_geom(dims);
  cudaStream_t st = state().stream;
  int status = WD_ERR_NOCONV, iters = 0, restarts = 0;
  double rel = 0.0;
  {
    Alloc al;
    const size_t V = 2 * (size_t)g.Vh;
    const size_t h32 = spinor_half_bytes(g, WD_F32), h64 = spinor_half_bytes(g, WD_F64);
    void *g32, *g64;
    NCK(al.get(&g32, gauge_bytes(g, WD_F32, 12)));
    NCK(al.get(&g64, gauge_bytes(g, WD_F64, 18)));
    const double* gd = gauge;
    if (!on_device(gauge)) {
      void* v;
      NCK(al.get(&v, 4 * V * 18 * sizeof(double)));
      NCK(cudaMemcpyAsync(v, gauge, 4 * V * 18 * sizeof(double), cudaMemcpyHostToDevice, st));
      gd = (const double*)v;
    }
    NCK(pack_gauge(g32, gd, g, WD_F32, 12, st));
    NCK(pack_gauge(g64, gd, g, WD_F64, 18, st));
#if WD_NN_FCG_BF16
    void* gbf = nullptr;  // the BF16 link copy of the network's layers
    if (wts) {
      NCK(al.get(&gbf, nn_gauge_bytes_bf16(g.Vh_pad)));
      NCK(nn_gauge_bf16(gbf, g32, g, st));
    }
#endif
    const double* bd = bsrc;
    double* canon = nullptr;
    {
      void* v;
      NCK(al.get(&v, V * 24 * sizeof(double)));
      canon = (double*)v;
    }
    if (!on_device(bsrc)) {
      NCK(cudaMemcpyAsync(canon, bsrc, V * 24 * sizeof(double), cudaMemcpyHostToDevice, st));
      bd = canon;
    }
    // FP64: b (full), x (full), bhat, r64 (even), t64 (odd); FP32 even
    // fields, and full-size buffers for the network's input and output
    // (their even halves are used)
    void *b64, *x64, *bhat, *r64, *t64, *r, *xs, *p, *q, *ts, *sA, *sB, *w, *z, *scal, *wa = nullptr;
    NCK(al.get(&b64, 2 * h64));
    NCK(al.get(&x64, 2 * h64));
    NCK(al.get(&bhat, h64));
    NCK(al.get(&r64, h64));
    NCK(al.get(&t64, h64));
    NCK(al.get(&r, h32));
    NCK(al.get(&xs, h32));
    NCK(al.get(&p, h32));
    NCK(al.get(&q, h32));
    NCK(al.get(&ts, h32));
    NCK(al.get(&sA, 2 * h32));
    NCK(al.get(&sB, 2 * h32));
    NCK(al.get(&w, 2 * h32));
    NCK(al.get(&z, 2 * h32));
    NCK(al.get(&scal, sizeof(FcgScalars)));
    FcgScalars* S = (FcgScalars*)scal;
    NnBuffers B;
    B.bytes8 = 2 * nn_half_bytes(g.Vh_pad, 8);
    if (wts) {
      NCK(al.get(&B.h1, B.bytes8));
      NCK(al.get(&B.h2, B.bytes8));
      NCK(al.get(&wa, NN_PARAMS * sizeof(float)));
      // N^+ = L1^+ L2^+ L3^+: the adjoint layers in reverse order have the
      // shapes of the forward layers (4 -> 8, 8 -> 8, 8 -> 4)
      float* WA = (float*)wa;
      nn_adjoint_weights<<<8, 256, 0, st>>>(wts + nn_layer_offset(2), WA + nn_layer_offset(0), 8, 4);
      nn_adjoint_weights<<<8, 256, 0, st>>>(wts + nn_layer_offset(1), WA + nn_layer_offset(1), 8, 8);
      nn_adjoint_weights<<<8, 256, 0, st>>>(wts + nn_layer_offset(0), WA + nn_layer_offset(2), 4, 8);
      NCK(cudaGetLastError());
    }
    int* flag = nullptr;
    NCK(device_flag(&flag, st));
    NCK(ensure_scratch((size_t)num_sms() * 8 * 4 + 2 * (size_t)((g.Vh + 127) / 128) + 1024));
    NCK(cudaMemsetAsync(scal, 0, sizeof(FcgScalars), st));
    NCK(pack_spinor(b64, bd, g, WD_FULL, WD_F64, st));
    NCK(norm2(&S->bn, b64, g, WD_F64, 2, st));
    NCK(cudaMemsetAsync(x64, 0, 2 * h64, st));
    NCK(cudaMemsetAsync(xs, 0, h32, st));
    const int grid = blas_grid(g.Vh, 256);
    RedScratch rs = scratch();
    FcgScalars hs;
    auto rd = [&]() -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(&hs, S, sizeof(hs), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return e;
      return cudaStreamSynchronize(st);
    };
    // one parity-restricted hopping launch: out = a H in + bx x + cy y
    auto hop = [&](int prec, int recon, const void* gauge_p, void* out, const void* in, int parity,
                   bool dagger, double a, const void* xf, double bx, const void* yf, double cy,
                   double* nrm) -> cudaError_t {
      DslashArgs d;
      d.out = out;
      d.in = in;
      d.gauge = gauge_p;
      d.a = a;
      d.x = xf;
      d.bx = bx;
      d.y = yf;
      d.cy = cy;
      d.norm_out = nrm;
      d.rs = rs;
      d.g = g;
      d.parity = parity;
      return launch_dslash(prec, d, recon, dagger, st);
    };
    // out = Mhat in (or Mhat^+) in FP32 on the even sites, ||out||^2 -> nrm
    auto mhat = [&](void* out, const void* in, bool dagger, double* nrm) -> cudaError_t {
      cudaError_t e = hop(WD_F32, 12, g32, ts, in, WD_ODD, dagger, 1.0, nullptr, 0.0, nullptr, 0.0,
                          nullptr);
      if (e != cudaSuccess) return e;
      return hop(WD_F32, 12, g32, out, ts, WD_EVEN, dagger, -kappa * kappa, in, 1.0, nullptr, 0.0,
                 nrm);
    };
    // z = N_e N_e^+ s (or z = s without a network), BF16 activations
    auto precond = [&](void* zo, const void* si) -> cudaError_t {
      if (!wts) return cudaMemcpyAsync(zo, si, h32, cudaMemcpyDeviceToDevice, st);
#if WD_NN_FCG_BF16
      cudaError_t e = nn_forward_bf16(g, gbf, (const float*)wa, si, w, B, flag, st, true);
      if (e != cudaSuccess) return e;
      return nn_forward_bf16(g, gbf, wts, w, zo, B, flag, st, true);
#else
      cudaError_t e = nn_forward_even(g, g32, (const float*)wa, si, w, B, flag, st);
      if (e != cudaSuccess) return e;
      return nn_forward_even(g, g32, wts, w, zo, B, flag, st);
#endif
    };
    // bhat = b_e + kappa H_eo b_o (FP64)
    NCK(hop(WD_F64, 18, g64, bhat, (const char*)b64 + h64, WD_EVEN, false, kappa, b64, 1.0,
            nullptr, 0.0, nullptr));
    void* s_cur = sA;
    void* s_old = sB;
    int kp = 0;
    // r64 = bhat - Mhat x64_e (FP64), r = r64, s = Mhat^+ r, z = N_e N_e^+ s, p = z
    auto restart = [&]() -> cudaError_t {
      cudaError_t e = hop(WD_F64, 18, g64, t64, x64, WD_ODD, false, 1.0, nullptr, 0.0, nullptr,
                          0.0, nullptr);
      if (e == cudaSuccess)
        e = hop(WD_F64, 18, g64, r64, t64, WD_EVEN, false, kappa * kappa, x64, -1.0, bhat, 1.0,
                &S->r64);
      if (e == cudaSuccess) e = convert_spinor(r, WD_F32, r64, WD_F64, g, 1, st);
      if (e == cudaSuccess) e = mhat(s_cur, r, true, nullptr);
      if (e == cudaSuccess) e = precond(z, s_cur);
      if (e != cudaSuccess) return e;
      fcg_dots<<<grid, 256, 0, st>>>((const char*)s_cur, nullptr, (const char*)z, S, kp, g, h32, 1,
                                     rs);
      fcg_update_p<<<grid, 256, 0, st>>>((char*)p, (const char*)z, S, kp, 1, g, h32, 1);
      return cudaGetLastError();
    };
    NCK(restart());
    NCK(rd());
    const double bnorm = std::sqrt(hs.bn);
    // the even-odd residual equals the full one up to rounding: aim a little lower
    const double target = P.tol * bnorm * 0.9;
    bool done = !(bnorm > 0) || std::sqrt(hs.r64) <= target;
    int since = 0;
    while (!done && iters < P.maxiter) {
      NCK(mhat(q, p, false, &S->qq[0]));
      fcg_update_xr<<<grid, 256, 0, st>>>((char*)xs, (char*)r, (const char*)p, (const char*)q, S,
                                         kp, g, h32, 1, rs);
      NCK(cudaGetLastError());
      iters++;
      since++;
      NCK(rd());
      const double rn = std::sqrt(hs.rr);
      if (!std::isfinite(rn)) {
        status = WD_ERR_NONFINITE;
        break;
      }
      if (rn <= target || since >= P.reliable_interval) {
        accumulate_full_kernel<<<grid, 256, 0, st>>>((char*)x64, (char*)xs, g, h64, h32, 1);
        NCK(cudaGetLastError());
        NCK(restart());
        NCK(rd());
        restarts++;
        since = 0;
        const double r64v = std::sqrt(hs.r64);
        if (!std::isfinite(r64v)) {
          status = WD_ERR_NONFINITE;
          break;
        }
        if (r64v <= target) done = true;
        continue;
      }
      std::swap(s_cur, s_old);
      NCK(mhat(s_cur, r, true, nullptr));
      NCK(precond(z, s_cur));
      fcg_dots<<<grid, 256, 0, st>>>((const char*)s_cur, (const char*)s_old, (const char*)z, S,
                                     1 - kp, g, h32, 1, rs);
      fcg_update_p<<<grid, 256, 0, st>>>((char*)p, (const char*)z, S, kp, 0, g, h32, 1);
      NCK(cudaGetLastError());
      kp ^= 1;
    }
    if (done) status = WD_OK;
    // the best iterate: x64_e (plus whatever accumulated since the last
    // reliable update), then x_o = b_o + kappa H_oe x_e, and the true
    // residual of the full system in FP64: r_e = b_e - x_e + kappa H_eo x_o
    // (the odd rows vanish up to rounding; they are computed as well)
    accumulate_full_kernel<<<grid, 256, 0, st>>>((char*)x64, (char*)xs, g, h64, h32, 1);
    NCK(cudaGetLastError());
    NCK(hop(WD_F64, 18, g64, (char*)x64 + h64, x64, WD_ODD, false, kappa, (const char*)b64 + h64,
            1.0, nullptr, 0.0, nullptr));
    {
      // true residual: ||b - D x||^2 from the FP64 full field r64f
      void* rf;
      NCK(al.get(&rf, 2 * h64));
      NCK(full_op(WD_F64, 18, g64, rf, x64, kappa, g, st, b64));
      NCK(norm2(&S->r64, rf, g, WD_F64, 2, st));
      NCK(rd());
      rel = bnorm > 0 ? std::sqrt(hs.r64) / bnorm : 0.0;
    }
    const bool xdev = on_device(x);
    double* xd = xdev ? x : canon;
    NCK(unpack_spinor(xd, x64, g, WD_FULL, WD_F64, st));
    if (!xdev) NCK(cudaMemcpyAsync(x, xd, V * 24 * sizeof(double), cudaMemcpyDeviceToHost, st));
    int hflag = 0;
    NCK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    NCK(cudaStreamSynchronize(st));
    if (hflag) status = WD_ERR_TIMEOUT;
    if (status == WD_OK && !(rel <= P.tol)) status = WD_ERR_NOCONV;
  }
  int fb_iters = 0;
  if (status != WD_OK) {
    // plain CG, the fallback: the even-odd mixed-precision solver from x
    wd_solve_params Q = P;
    Q.use_initial_guess = 1;
    Q.solver = WD_SOLVER_CG;
    Q.maxiter = 100000;
    wd_solve_info fi;
    std::memset(&fi, 0, sizeof(fi));
    status = solve_impl(x, bsrc, gauge, kappa, dims, &Q, &fi);
    fb_iters = fi.iters;
    rel = fi.true_residual;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = iters + fb_iters;
    info->reliable_updates = restarts;
    info->status = status;
    info->true_residual = rel;
    info->fallback_iters = fb_iters;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

}  // namespace wd
