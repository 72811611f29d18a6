// wd_dslash_ex_noalloc: the fused hopping kernel of wd_dslash_ex, with the
// scratch of its FP64 norm reduction taken from a fixed array compiled into
// this library instead of memory the library allocates at run time.
//
// Some callers cannot let a library call cudaMalloc:
//  * code that records its launches into a CUDA graph by stream capture
//    (an allocation in the middle of a capture is not allowed and breaks it);
//  * applications whose device memory is owned by another allocator, e.g. a
//    framework caching allocator that has already reserved the GPU;
//  * latency-critical loops that must never trigger the device-wide
//    synchronisation that growing a cudaMalloc'd buffer (cudaFree) implies.
// For them this entry point allocates nothing: the per-CTA partial sums of
// the deterministic reduction (summed by the launch that follows the hopping
// kernel) live in `g_noalloc_scratch` below, which every GPU that loads the
// library holds until the process exits.
#include <cstdint>

#include "wd_internal.h"

namespace {

// One partial per 128-site CTA: 16384 partials cover V/2 <= 2,097,152 sites
// (e.g. 32^3x128).
constexpr int kMaxPartials = 16384;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kMaxPartials];

// Device address of g_noalloc_scratch per device, looked up once.  In host
// code the symbol's name is only a host-side stand-in, never a device address.
double* g_scratch_addr[kMaxDevices] = {nullptr};

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

using namespace wd;

extern "C" int wd_dslash_ex_noalloc(void* out, const void* in, const void* gauge, int parity,
                                    int dagger, double a, const void* x, double bx,
                                    const void* y, double cy, double* norm2, const int dims[4],
                                    int prec, int recon) {
  // ---- validation, all on the host, before any CUDA call ----
  // the flag bits of wd_dslash_ex: temporal-gauge links, staged neighbours
  const int tg = (recon & WD_TEMPORAL_GAUGE_BIT) != 0;
  const int staged = (recon & WD_STAGE_NEIGHBOURS) != 0;
  recon &= ~(WD_TEMPORAL_GAUGE_BIT | WD_STAGE_NEIGHBOURS);
  if (!dims) return WD_ERR_NULL;
  long long V = 1;
  for (int i = 0; i < 4; i++) {
    if (dims[i] < 2 || (dims[i] & 1)) return WD_ERR_DIMS;
    V *= dims[i];
    if (V > (1LL << 30)) return WD_ERR_DIMS;
  }
  if (prec < WD_F64 || prec > WD_F16) return WD_ERR_PREC;
  if (!out || !in || !gauge) return WD_ERR_NULL;
  if (!aligned16(out) || !aligned16(in) || !aligned16(gauge) || (x && !aligned16(x)) ||
      (y && !aligned16(y)) || (norm2 && ((uintptr_t)norm2 & 7u)))
    return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD) return WD_ERR_ARG;
  if (link_bytes(prec, recon) == 0) return WD_ERR_PREC;
  if (out == in) return WD_ERR_ALIAS;
  const Geom g = make_geom(dims);
  const long long ctas = (g.Vh + DSLASH_BS - 1) / DSLASH_BS;
  if (ctas > kMaxPartials) return WD_ERR_SCRATCH;
  if (staged && (prec != WD_F16 || recon != 12 || tg || norm2 || (g.S2 & 31) != 0))
    return WD_ERR_ARG;
  cudaStream_t st = state().stream;
  if (staged) {
    // no reduction, hence no scratch: the staged kernel's fault flag is a
    // __device__ variable of the library as well
    DslashArgs d;
    d.out = out;
    d.in = in;
    d.gauge = gauge;
    d.x = x;
    d.y = y;
    d.a = a;
    d.bx = bx;
    d.cy = cy;
    d.norm_out = nullptr;
    d.rs = RedScratch{};
    d.g = g;
    d.parity = parity;
    cudaError_t es = launch_dslash_f16_staged(d, recon, dagger != 0, state().wait_limit, st);
    if (es != cudaSuccess) {
      state().last_cuda_error = (int)es;
      return WD_ERR_CUDA;
    }
    return WD_OK;
  }

  // ---- once per device: the device address of the fixed scratch ----
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    state().last_cuda_error = (int)e;
    return WD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return WD_ERR_ARG;
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      state().last_cuda_error = (int)e;
      return WD_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  RedScratch rs;
  rs.partials = g_scratch_addr[dev];
  rs.counter = nullptr;  // (the hopping kernels' reductions use no counter)
  DslashArgs d;
  d.out = out;
  d.in = in;
  d.gauge = gauge;
  d.x = x;
  d.y = y;
  d.a = a;
  d.bx = bx;
  d.cy = cy;
  d.norm_out = norm2;
  d.rs = rs;
  d.g = g;
  d.parity = parity;
  d.tg = tg;
  d.no_tune = 1;  // the CTA size tuner allocates: use the tuned or default size
  e = launch_dslash(prec, d, recon, dagger != 0, st);
  if (e != cudaSuccess) {
    state().last_cuda_error = (int)e;
    return WD_ERR_CUDA;
  }
  return WD_OK;
}
