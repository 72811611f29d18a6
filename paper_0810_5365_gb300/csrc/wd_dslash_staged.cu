// FP16 hopping kernel with the far neighbours staged in shared memory by the
// bulk-copy (TMA) engine.
//
// With the site-blocked layout, a block of 32 checkerboard sites whose sites
// all lie in one (z, t) slice of the lattice (L0 L1 / 2 a multiple of 32) has
// its +z, -z, +t and -t neighbours in four whole 32-site blocks of the other
// parity's field: the same lane of the block one z- or t-stride away (with
// the periodic wrap applied to the block index).  In the FP16 format such a
// block is one contiguous 1536-byte span (three planes of 32 x 16 bytes), so
// each warp stages its four far neighbour blocks with four cp.async.bulk
// copies issued by one lane and completed on the warp's own mbarrier.  The
// copies run while the warp computes its x and y hops from global memory
// (near neighbours, mostly L1 hits); the z and t hops then read their
// spinors from shared memory.  The eight neighbour scales are needed before
// the first hop (the hops accumulate relative to the largest) and are loaded
// directly, as are the links, which are used once per application.
//
// Each warp's mbarrier is used once (phase 0).  The wait is bounded: if it
// gives up after `spin_limit` polls, the kernel raises the device's fault
// flag, drains its copies with a second, much longer bounded wait and writes
// NaN to that warp's sites, so that the failure shows in any later norm,
// solve or check of the output.  A raised flag marks the whole launch (and
// any launch since the flag was last read) as untrustworthy, not only the
// poisoned sites: should even the drain wait give up, the warp exits with a
// copy possibly still writing into shared memory that the next CTA on that
// SM may own.
#include "wd_dslash.cuh"
#include "wd_tc.cuh"

namespace wd {

namespace {

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16), completing `bytes` of transaction count on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

constexpr int STG_WARPS = 4;           // CTA = 4 site blocks = 128 sites
constexpr uint32_t STG_SPAN = 1536;    // bytes of one FP16 site block (3 x 32 x 16)
// polls of the drain wait after a timeout: about 7 s at some 100 ns per poll,
// far beyond any copy of 6.5 KB
constexpr long STG_DRAIN_LIMIT = 1L << 26;

// Fault flag of the asynchronous bounded waits, one per device (a __device__
// variable exists once in every GPU context that loads the library), raised
// by a timed-out staged launch and read and cleared by stage_fault_take().
__device__ int g_stage_fault;

struct __align__(16) StageWarp {
  int4 sp[4][3][32];  // [z+, z-, t+, t-][plane][lane]
};

// the link of a hop whose spinor comes from shared memory
__device__ __forceinline__ void fetch_link_f16(RawF16& r, const void* __restrict__ gauge,
                                               int region, int lcb, int VP) {
  r.la = __ldg((const int4*)gauge + (size_t)region * VP + lcb);
  r.lb = __ldg((const int2*)((const char*)gauge + (size_t)8 * VP * 16) + (size_t)region * VP +
               lcb);
}

template <bool DAG>
__global__ void __launch_bounds__(STG_WARPS * 32, DslashMinBlocks<WD_F16, false>::value)
    dslash_f16_staged_kernel(const DslashArgs a, long spin_limit) {
  __shared__ StageWarp stage[STG_WARPS];
  __shared__ uint64_t bar[STG_WARPS];
  pdl_begin();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Geom& g = a.g;
  const int blk = blockIdx.x * STG_WARPS + warp;
  if (blk * 32 >= g.Vh) return;  // whole warps only: Vh is a multiple of 32
  const int cb = blk * 32 + lane;
  const int p = a.parity, q = 1 - p, VP = g.Vh_pad;
  int x0, x1, x2, x3;
  cb_coords(cb, p, g, x0, x1, x2, x3);  // x2 and x3 are the same in the whole warp

  // far neighbour blocks (uniform in the warp)
  const int zs = g.S2 >> 5, ts = g.S3 >> 5;
  const int bzf = x2 == g.L[2] - 1 ? blk - (g.L[2] - 1) * zs : blk + zs;
  const int bzb = x2 == 0 ? blk + (g.L[2] - 1) * zs : blk - zs;
  const int btf = x3 == g.L[3] - 1 ? blk - (g.L[3] - 1) * ts : blk + ts;
  const int btb = x3 == 0 ? blk + (g.L[3] - 1) * ts : blk - ts;
  StageWarp& s = stage[warp];
  if (lane == 0) {
    mbar_init(&bar[warp], 1);
    mbar_fence_init();
    fence_smem_to_async();
    mbar_arrive_expect_tx(&bar[warp], 4 * STG_SPAN);
    const char* sp = (const char*)a.in;
    const int nb[4] = {bzf, bzb, btf, btb};
#pragma unroll
    for (int d = 0; d < 4; d++)
      bulk_g2s(&s.sp[d][0][0], sp + (size_t)nb[d] * STG_SPAN, STG_SPAN, &bar[warp]);
  }
  __syncwarp();  // the barrier is initialised before any lane polls it

  const int row = cb - (x0 >> 1);
  const int f0 = row + ((x0 + 1 == g.L[0] ? 0 : x0 + 1) >> 1);
  const int b0 = row + ((x0 == 0 ? g.L[0] - 1 : x0 - 1) >> 1);
  const int f1 = x1 == g.L[1] - 1 ? cb - (g.L[1] - 1) * g.S1 : cb + g.S1;
  const int b1 = x1 == 0 ? cb + (g.L[1] - 1) * g.S1 : cb - g.S1;
  // sites of the far neighbours (the same lane of the neighbour blocks),
  // also the sites of the backward z and t links
  const int f2 = bzf * 32 + lane, b2 = bzb * 32 + lane;
  const int f3 = btf * 32 + lane, b3 = btb * 32 + lane;
  const bool fflip = x3 == g.L[3] - 1;
  const bool bflip = x3 == 0;
  constexpr int SF = DAG ? -1 : 1;
  constexpr int SB_ = -SF;

  cx<float> acc[12];
  bool stored = false;
  // the eight neighbour scales first, then the near hops from global memory
  // with two hops of loads in flight (the same arithmetic, in the same
  // order, as the unstaged kernel's hops_f16)
  {
    const float* scl = (const float*)((const char*)a.in + (size_t)VP * 48);
    float sc[8] = {__ldg(scl + f0), __ldg(scl + b0), __ldg(scl + f1), __ldg(scl + b1),
                   __ldg(scl + f2), __ldg(scl + b2), __ldg(scl + f3), __ldg(scl + b3)};
    __half2 ah[12];
#pragma unroll
    for (int k = 0; k < 12; k++) ah[k] = __float2half2_rn(0.f);
    RawF16 r0 = fetch_f16(a.in, a.gauge, f0, 0 + p, cb, VP);
    RawF16 r1 = fetch_f16(a.in, a.gauge, b0, 0 + q, b0, VP);
    RawF16 r2 = fetch_f16(a.in, a.gauge, f1, 2 + p, cb, VP);
    __half2 rel[4];
    const float smax = f16_rel(sc, fflip, bflip, rel);
    compute_f16<0, SF, true>(ah, r0, __low2half2(rel[0]));
    RawF16 r3 = fetch_f16(a.in, a.gauge, b1, 2 + q, b1, VP);
    compute_f16<0, SB_, false>(ah, r1, __high2half2(rel[0]));
    fetch_link_f16(r0, a.gauge, 4 + p, cb, VP);
    fetch_link_f16(r1, a.gauge, 4 + q, b2, VP);
    compute_f16<1, SF, true>(ah, r2, __low2half2(rel[1]));
    fetch_link_f16(r2, a.gauge, 6 + p, cb, VP);
    compute_f16<1, SB_, false>(ah, r3, __high2half2(rel[1]));
    fetch_link_f16(r3, a.gauge, 6 + q, b3, VP);
    // far hops from shared memory
    if (mbar_wait_bounded(&bar[warp], 0, spin_limit)) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        r0.s[k] = s.sp[0][k][lane];
        r1.s[k] = s.sp[1][k][lane];
      }
      compute_f16<2, SF, true>(ah, r0, __low2half2(rel[2]));
      compute_f16<2, SB_, false>(ah, r1, __high2half2(rel[2]));
#pragma unroll
      for (int k = 0; k < 3; k++) {
        r2.s[k] = s.sp[2][k][lane];
        r3.s[k] = s.sp[3][k][lane];
      }
      compute_f16<3, SF, true>(ah, r2, __low2half2(rel[3]));
      compute_f16<3, SB_, false>(ah, r3, __high2half2(rel[3]));
      const float kf = (float)a.a * smax;
      if (!a.x && !a.y) {
        store_f16_h2(a.out, cb, VP, ah, kf, acc);
        stored = true;
      } else {
        f16_widen(acc, ah, kf);
      }
    } else {
      if (lane == 0) atomicExch(&g_stage_fault, 1);
      // the copies may still be in flight: drain them (bounded, long) before
      // the CTA's shared memory is released
      mbar_wait_bounded(&bar[warp], 0, STG_DRAIN_LIMIT);
      // the output of these sites is poisoned (NaN), so that the failure
      // reaches any later norm, solve or check of the result
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = mk<float>(__int_as_float(0x7fc00000), 0.f);
    }
  }

  if (stored) return;
  if (a.x) {
    cx<float> v[12];
    load_spinor_rw<WD_F16, float>(v, a.x, cb, VP);
    const float cbx = (float)a.bx;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      acc[k].r = fmaf(cbx, v[k].r, acc[k].r);
      acc[k].i = fmaf(cbx, v[k].i, acc[k].i);
    }
  }
  if (a.y) {
    cx<float> v[12];
    load_spinor_rw<WD_F16, float>(v, a.y, cb, VP);
    const float ccy = (float)a.cy;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      acc[k].r = fmaf(ccy, v[k].r, acc[k].r);
      acc[k].i = fmaf(ccy, v[k].i, acc[k].i);
    }
  }
  store_spinor<WD_F16, float>(a.out, cb, VP, acc);
}

}  // namespace

namespace {
constexpr int kMaxDevices = 64;
bool g_carveout_set[kMaxDevices] = {false};
}  // namespace

// The staged kernel covers FP16 fields with 12-real links, no temporal gauge
// and no fused reduction, on lattices whose (z, t) slices hold a multiple of
// 32 sites of one parity; cudaErrorNotSupported otherwise.  spin_limit: polls
// of the bounded wait for the copies (0 gives up at once).  Allocates nothing.
cudaError_t launch_dslash_f16_staged(const DslashArgs& a, int recon, bool dagger, long spin_limit,
                                     cudaStream_t st) {
  const Geom& g = a.g;
  if (recon != 12 || a.tg || a.norm_out || (g.S2 & 31) != 0 || spin_limit < 0)
    return cudaErrorNotSupported;
  const int nblk = g.Vh / 32;
  dim3 grid((nblk + STG_WARPS - 1) / STG_WARPS), block(STG_WARPS * 32);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // the carveout is a per-device function attribute: set it once per device
  if (dev >= 0 && dev < kMaxDevices && !g_carveout_set[dev]) {
    // shared memory for the register budget's CTAs per SM and no more: the
    // rest of the unified L1 keeps serving the near neighbours and links
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const long need = (long)DslashMinBlocks<WD_F16, false>::value *
                      (long)(sizeof(StageWarp) * STG_WARPS + 64);
    int pct = smem_sm > 0 ? (int)((100 * need + smem_sm - 1) / smem_sm) : 100;
    pct = pct > 100 ? 100 : pct;
    cudaFuncSetAttribute(dslash_f16_staged_kernel<false>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    cudaFuncSetAttribute(dslash_f16_staged_kernel<true>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    cudaGetLastError();
    g_carveout_set[dev] = true;
  }
  if (dagger) return launch_pdl(dslash_f16_staged_kernel<true>, grid, block, st, a, spin_limit);
  return launch_pdl(dslash_f16_staged_kernel<false>, grid, block, st, a, spin_limit);
}

// Read and clear the current device's fault flag after the work queued on
// `st` has finished (synchronises st).  *fault = 1 if a staged launch gave up
// waiting since the flag was last cleared.  Allocates nothing.
cudaError_t stage_fault_take(int* fault, cudaStream_t st) {
  int h = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_stage_fault, sizeof(int), 0,
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && h) {
    static const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_stage_fault, &zero, sizeof(int), 0, cudaMemcpyHostToDevice,
                                st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  *fault = h;
  return e;
}

}  // namespace wd
