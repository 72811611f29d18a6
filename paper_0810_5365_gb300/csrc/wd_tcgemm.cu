// A plain BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores, one
// 128-row tile per CTA: operands staged in shared memory (K-major, no
// swizzle), tcgen05.mma issued by one thread with the accumulator in TMEM,
// completion through an mbarrier, and the result read back with tcgen05.ld.
// It exposes, on its own, the contraction core that the learned
// preconditioner's layers use, so the tests can pin the descriptor and
// operand layouts against a host GEMM.
#include <cuda_bf16.h>

#include "wd_internal.h"
#include "wd_tc.cuh"

namespace wd {

constexpr long TC_SPIN_LIMIT = 1L << 22;

// D[M x N] = A[M x K] * B[K x N], row-major, BF16 in, FP32 out.
// M % 128 == 0, K % 16 == 0, K <= 256, N % 16 == 0, 16 <= N <= 256.
__global__ void __launch_bounds__(128) tc_gemm_kernel(const __nv_bfloat16* __restrict__ A,
                                                      const __nv_bfloat16* __restrict__ B,
                                                      float* __restrict__ D, int K, int N,
                                                      int* err) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  unsigned char* sa = sm;                        // 128 x K
  unsigned char* sb = sm + (size_t)128 * K * 2;  // N x K (B transposed)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;

  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, ncols);
    tmem_relinquish();
  }
  for (int e = tid; e < 128 * K; e += 128) {
    const int r = e / K, k = e - r * K;
    *(__nv_bfloat16*)(sa + kmajor_offset(r, k, K)) = A[(size_t)(m0 + r) * K + k];
  }
  for (int e = tid; e < N * K; e += 128) {
    const int k = e / N, n = e - k * N;
    *(__nv_bfloat16*)(sb + kmajor_offset(n, k, K)) = B[(size_t)k * N + n];
  }
  fence_smem_to_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = make_idesc_bf16(128, N);
    const uint32_t sbo = (uint32_t)(K / 8) * 128;
    for (int s = 0; s < K / 16; s++) {
      const uint64_t ad = make_smem_desc(smem_u32(sa) + s * 256, 128, sbo);
      const uint64_t bd = make_smem_desc(smem_u32(sb) + s * 256, 128, sbo);
      tc_mma_bf16(tbase, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc_commit(&bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0, TC_SPIN_LIMIT);
  if (!ok && lane == 0) atomicExch(err, 1);
  tc_fence_after();
  if (ok) {
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
      float* drow = D + (size_t)(m0 + 32 * warp + lane) * N + c;
#pragma unroll
      for (int i = 0; i < 16; i++) drow[i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, ncols);
}

cudaError_t tc_gemm_bf16(const void* A, const void* B, float* D, int M, int K, int N, int* err,
                         cudaStream_t st) {
  const size_t smem = (size_t)128 * K * 2 + (size_t)N * K * 2;  // <= 192 KB
  static size_t attr = 0;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  tc_gemm_kernel<<<M / 128, 128, smem, st>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, D,
                                             K, N, err);
  return cudaGetLastError();
}

// The bounded-wait failure path, exercised on purpose: one warp initialises
// an mbarrier that nothing ever arrives on and waits for its first phase with
// the same bounded helper as the tensor-core kernels.  When the polls run out
// it raises the device error flag, as those kernels do, and returns normally.
__global__ void wait_selftest_kernel(long spins, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, spins);
  if (threadIdx.x == 0 && !ok) atomicExch(err, 1);
}

cudaError_t wait_selftest(long spins, int* err, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(spins, err);
  return cudaGetLastError();
}

}  // namespace wd
