// Host-side internals of libwd shared by its translation units.
#pragma once

#include <cuda_runtime.h>

#include "wd_common.cuh"

namespace wd {

// threads per block of the hopping kernel, and the minimum number of its
// blocks per SM that the register allocation must allow
#ifndef WD_DSLASH_BS
#define WD_DSLASH_BS 128
#endif
// Register budgets from sweeps on GB300 (32^3x64): FP32 is fastest with 7
// resident 128-thread blocks per SM (<= 72 registers), FP16 with 6 (<= 80
// registers, two hops of loads in flight; 5 and 7 are slower); FP64 is
// bound by its arithmetic pipe and gets 3 (168 registers, no spills).
#ifndef WD_DSLASH_MINB_F64
#define WD_DSLASH_MINB_F64 3
#endif
#ifndef WD_DSLASH_MINB_F32
#define WD_DSLASH_MINB_F32 7
#endif
#ifndef WD_DSLASH_MINB_F32_NORM
#define WD_DSLASH_MINB_F32_NORM 6
#endif
#ifndef WD_DSLASH_MINB_F16
#define WD_DSLASH_MINB_F16 6
#endif
constexpr int DSLASH_BS = WD_DSLASH_BS;
// (the fused-norm FP32 variant needs 80 registers to stay free of spills)
template <int P, bool NORM>
struct DslashMinBlocks {
  // (one fewer block for FP32 kernels that reduce, see the sweep above)
  static constexpr int value =
      P == WD_F64   ? WD_DSLASH_MINB_F64
      : P == WD_F32 ? (NORM ? WD_DSLASH_MINB_F32_NORM : WD_DSLASH_MINB_F32)
                    : WD_DSLASH_MINB_F16;
};

struct DslashArgs {
  void* out;
  const void* in;
  const void* gauge;
  const void* x;     // optional (may alias out)
  const void* y;     // optional (may alias out)
  double a, bx, cy;
  double* norm_out;  // ||out||^2 when the kernel reduces
  RedScratch rs;
  Geom g;
  int parity;        // parity of the output sites
  int tg = 0;        // links in temporal gauge: U_t = 1 off the last time slice
  // reduction fused into the epilogue when norm_out != nullptr:
  //   RED_NORM       norm_out[0]    = ||out||^2
  //   RED_NORM_DOTX  norm_out[0..2] = ||out||^2, <out, x> (re, im)
  //   RED_DOTZ       norm_out[0..1] = <z, out>   (re, im),  <a, b> = sum conj(a) b
  int red_mode = 1;
  const void* z = nullptr;
  // 1: never time launch shapes for this call (it must not allocate)
  int no_tune = 0;
};

// the run-time tuners (wd_batch.cu): on/off switch, a forced CTA size of the
// single-field hopping kernel (0: tuned), and the report lines of its choices
int autotune_enabled();
int dslash_forced_block();
void dslash_tune_record(const char* line);
// 1: hopping kernels are launched as programmatic dependent launches
int launch_overlap();
int set_launch_overlap(int enable);

// Launch kernel k (which starts with pdl_begin) with launch overlap on
// (wd_set_launch_overlap) as a programmatic dependent launch, else as a
// plain stream-ordered launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = launch_overlap() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

enum { RED_NONE = 0, RED_NORM = 1, RED_NORM_DOTX = 2, RED_DOTZ = 3 };

// bit OR-ed into a `recon` argument: the gauge field is in temporal gauge
// (time links are the identity except on the slice t = L3-1), so the hopping
// kernels skip those links' loads and mat-vecs
constexpr int WD_TEMPORAL_GAUGE_BIT = 0x100;

cudaError_t launch_dslash_f64(const DslashArgs& a, int recon, bool dagger, cudaStream_t st);
cudaError_t launch_dslash_f32(const DslashArgs& a, int recon, bool dagger, cudaStream_t st);
cudaError_t launch_dslash_f16(const DslashArgs& a, int recon, bool dagger, cudaStream_t st);

// FP16 hopping with the +-z, +-t neighbours staged in shared memory by bulk
// copies (wd_dslash_staged.cu); spin_limit bounds the wait for the copies.
// A launch whose wait gave up raises the device's fault flag, which
// stage_fault_take reads and clears (after synchronising st).  Neither
// allocates.
cudaError_t launch_dslash_f16_staged(const DslashArgs& a, int recon, bool dagger,
                                     long spin_limit, cudaStream_t st);
cudaError_t stage_fault_take(int* fault, cudaStream_t st);

inline cudaError_t launch_dslash(int prec, const DslashArgs& a, int recon, bool dagger,
                                 cudaStream_t st) {
  switch (prec) {
    case WD_F64: return launch_dslash_f64(a, recon, dagger, st);
    case WD_F32: return launch_dslash_f32(a, recon, dagger, st);
    case WD_F16: return launch_dslash_f16(a, recon, dagger, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// library state
// ---------------------------------------------------------------------------

struct State {
  cudaStream_t stream = nullptr;
  int last_cuda_error = 0;
  // reduction scratch shared by every reducing kernel; kernels on one stream
  // run in order, so one set suffices (calls that overlap on the GPU race)
  double* partials = nullptr;
  unsigned* counter = nullptr;
  size_t partials_cap = 0;  // doubles
  int num_sms = 0;
  int* dev_flag = nullptr;  // device int: set by kernels whose bounded waits gave up
  // polls of the first bounded wait of the asynchronous kernels (wd_set_wait_limit)
  long wait_limit = 1L << 22;
};

State& state();

// grow the reduction scratch to hold `doubles` partial sums (not during capture)
cudaError_t ensure_scratch(size_t doubles);
RedScratch scratch();
// out[j] = sum over b < nblocks of partials[b * n + j] (j < n, n = 1, 2 or 3),
// in block order: the cross-block step of the kernels that leave per-block
// partials (block_partials); one CTA, launched with launch_pdl.  SumOut: a
// destination per j (null: not written).
struct SumOut {
  double* p[3];
};
cudaError_t sum_block_partials(int n, const double* partials, int nblocks, SumOut out,
                               cudaStream_t st);
cudaError_t sum_block_partials(int n, const double* partials, int nblocks, double* out,
                               cudaStream_t st);
int num_sms();

// grid of the grid-stride BLAS/reduction kernels for n sites
int blas_grid(long long n, int bs);

// ---------------------------------------------------------------------------
// layout and BLAS (wd_blas.cu)
// ---------------------------------------------------------------------------

cudaError_t pack_spinor(void* dst, const double* src, const Geom& g, int parity, int prec,
                        cudaStream_t st);
cudaError_t unpack_spinor(double* dst, const void* src, const Geom& g, int parity, int prec,
                          cudaStream_t st);
cudaError_t pack_gauge(void* dst, const double* src, const Geom& g, int prec, int recon,
                       cudaStream_t st);
// nh = 1 (one parity) or 2 (both halves, laid out even then odd)
cudaError_t convert_spinor(void* dst, int dprec, const void* src, int sprec, const Geom& g,
                           int nh, cudaStream_t st);
cudaError_t norm2(double* res, const void* x, const Geom& g, int prec, int nh, cudaStream_t st);
cudaError_t cdot(double* res, const void* x, const void* y, const Geom& g, int prec, int nh,
                 cudaStream_t st);
cudaError_t axpby(double a, const void* x, double b, void* y, const Geom& g, int prec, int nh,
                  cudaStream_t st);

// zeroed device flag for bounded device-side waits (allocated on first use)
cudaError_t device_flag(int** flag, cudaStream_t st);

// tensor-core GEMM (wd_tcgemm.cu)
cudaError_t tc_gemm_bf16(const void* A, const void* B, float* D, int M, int K, int N, int* err,
                         cudaStream_t st);

// temporal gauge (wd_gauge.cu): canonical FP64 fields on the device
cudaError_t gauge_fix_temporal(double* Uout, double* omega, const double* Uin, const Geom& g,
                               cudaStream_t st);
cudaError_t rotate_spinor(double* out, const double* in, const double* omega, const Geom& g,
                          int dagger, cudaStream_t st);

}  // namespace wd
