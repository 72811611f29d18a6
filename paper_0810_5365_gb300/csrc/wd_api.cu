// The extern "C" entry points of libwd (declared and documented in
// include/wd.h): argument validation, status codes, and dispatch to the
// kernels.  No C++ exception crosses this boundary.
#include <cstdint>
#include <cstring>

#include "wd_internal.h"

namespace wd {
int nn_apply_impl(void* out, const void* in, const float* w, const void* gauge, const int dims[4]);
int nn_init_impl(float* w_dev, double kappa);
int nn_apply_ex_impl(void* out, const void* in, const float* w, const void* gauge,
                     const int dims[4], int flags);
int nn_layer_impl(void* out, const void* in, const float* w, int cin, int cout, const void* gauge,
                  const int dims[4]);
int gaussian_spinor_impl(void* out, unsigned long long seed, unsigned long long stream,
                         unsigned long long first, const int dims[4]);
int nn_wgrad_impl(float* grad, const void* in, const void* delta, int cin, int cout,
                  const void* gauge, const int dims[4]);
int nn_train_impl(float* w, const double* gauge, double kappa, const int dims[4],
                  const wd_nn_train_params* prm, wd_nn_train_info* info);
int fgcr_impl(double* x, const double* bsrc, const double* gauge, double kappa,
              const int dims[4], const float* wts, const wd_solve_params* prm,
              wd_solve_info* info, int m);
int fcg_impl(double* x, const double* bsrc, const double* gauge, double kappa, const int dims[4],
             const float* wts, const wd_solve_params* prm, wd_solve_info* info);
int solve_batch_impl(const wd_batch_problem* probs, int nprob, const wd_solve_params* prm,
                     wd_solve_info* infos);
cudaError_t dslash_mrhs(void* out, const void* in, const void* gauge, int parity, int dagger,
                        double a, const void* x, double bx, int nrhs, double* norms,
                        const Geom& g, int prec, int recon, cudaStream_t st);
int solve_impl(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
               const wd_solve_params* prm, wd_solve_info* info);
void solver_finalize();
cudaError_t wait_selftest(long spins, int* err, cudaStream_t st);
int set_autotune(int enable);
int set_batch_mode(int mode);
int dslash_set_block(int bs);
int mrhs_set_lanes(int lanes);
int tune_report(char* buf, size_t len);
}  // namespace wd

using namespace wd;

namespace {
// Entry points whose implementations use host containers run through this
// guard, so that a host allocation failure becomes a status (WD_ERR_CUDA with
// cudaErrorMemoryAllocation) instead of an exception crossing the C ABI.
template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (...) {
    state().last_cuda_error = (int)cudaErrorMemoryAllocation;
    return WD_ERR_CUDA;
  }
}
}  // namespace


namespace {

int check_dims(const int* dims) {
  if (!dims) return WD_ERR_NULL;
  long long V = 1;
  for (int i = 0; i < 4; i++) {
    if (dims[i] < 2 || (dims[i] & 1)) return WD_ERR_DIMS;
    V *= dims[i];
    if (V > (1LL << 30)) return WD_ERR_DIMS;  // checkerboard indices stay in int32
  }
  return WD_OK;
}

bool aligned(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_prec(int prec) { return (prec >= WD_F64 && prec <= WD_F16) ? WD_OK : WD_ERR_PREC; }

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return WD_OK;
  state().last_cuda_error = (int)e;
  return WD_ERR_CUDA;
}

#define WD_TRY(expr)            \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != WD_OK) return rc_; \
  } while (0)

}  // namespace

extern "C" {

int wd_set_stream(void* s) {
  state().stream = (cudaStream_t)s;
  return WD_OK;
}

void* wd_get_stream(void) { return (void*)state().stream; }

const char* wd_error_string(int status) {
  switch (status) {
    case WD_OK: return "WD_OK";
    case WD_ERR_NULL: return "WD_ERR_NULL: a required pointer is NULL";
    case WD_ERR_DIMS: return "WD_ERR_DIMS: every extent must be even and >= 2";
    case WD_ERR_PREC: return "WD_ERR_PREC: unknown or unsupported precision / link format";
    case WD_ERR_ALIGN: return "WD_ERR_ALIGN: device buffers must be 16-byte aligned";
    case WD_ERR_ALIAS: return "WD_ERR_ALIAS: output aliases an input read at neighbour sites";
    case WD_ERR_NOCONV: return "WD_ERR_NOCONV: solver did not reach the tolerance";
    case WD_ERR_NONFINITE: return "WD_ERR_NONFINITE: NaN or Inf in a residual";
    case WD_ERR_TIMEOUT: return "WD_ERR_TIMEOUT: a bounded device wait gave up";
    case WD_ERR_CUDA: return "WD_ERR_CUDA: a CUDA runtime call failed";
    case WD_ERR_ARG: return "WD_ERR_ARG: argument out of range";
    case WD_ERR_BREAKDOWN: return "WD_ERR_BREAKDOWN: Krylov breakdown";
    case WD_ERR_SCRATCH:
      return "WD_ERR_SCRATCH: lattice exceeds the fixed scratch of wd_dslash_ex_noalloc "
             "(V/2 <= 2097152 sites)";
  }
  return "unknown status";
}

int wd_last_cuda_error(void) { return state().last_cuda_error; }

void wd_finalize(void) {
  cudaDeviceSynchronize();
  solver_finalize();
  State& s = state();
  if (s.partials) cudaFree(s.partials);
  if (s.counter) cudaFree(s.counter);
  if (s.dev_flag) cudaFree(s.dev_flag);
  s.partials = nullptr;
  s.counter = nullptr;
  s.dev_flag = nullptr;
  s.partials_cap = 0;
}

size_t wd_spinor_bytes(const int dims[4], int parity, int prec) {
  if (check_dims(dims) != WD_OK || check_prec(prec) != WD_OK) return 0;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return 0;
  Geom g = make_geom(dims);
  size_t h = spinor_half_bytes(g, prec);
  return parity == WD_FULL ? 2 * h : h;
}

size_t wd_gauge_bytes(const int dims[4], int prec, int recon) {
  if (check_dims(dims) != WD_OK || check_prec(prec) != WD_OK) return 0;
  if (link_bytes(prec, recon) == 0) return 0;
  return gauge_bytes(make_geom(dims), prec, recon);
}

int wd_pack_gauge(void* dst, const double* src, const int dims[4], int prec, int recon) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!dst || !src) return WD_ERR_NULL;
  if (!aligned(dst) || !aligned(src)) return WD_ERR_ALIGN;
  if (link_bytes(prec, recon) == 0) return WD_ERR_PREC;
  return cuda_status(pack_gauge(dst, src, make_geom(dims), prec, recon, state().stream));
}

int wd_pack_spinor(void* dst, const double* src, const int dims[4], int parity, int prec) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!dst || !src) return WD_ERR_NULL;
  if (!aligned(dst) || !aligned(src)) return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return WD_ERR_ARG;
  return cuda_status(pack_spinor(dst, src, make_geom(dims), parity, prec, state().stream));
}

int wd_unpack_spinor(double* dst, const void* src, const int dims[4], int parity, int prec) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!dst || !src) return WD_ERR_NULL;
  if (!aligned(dst) || !aligned(src)) return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return WD_ERR_ARG;
  return cuda_status(unpack_spinor(dst, src, make_geom(dims), parity, prec, state().stream));
}

int wd_convert_spinor(void* dst, int dst_prec, const void* src, int src_prec, const int dims[4],
                      int parity) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(dst_prec));
  WD_TRY(check_prec(src_prec));
  if (!dst || !src) return WD_ERR_NULL;
  if (!aligned(dst) || !aligned(src)) return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return WD_ERR_ARG;
  if (dst == src && dst_prec != src_prec) return WD_ERR_ALIAS;
  return cuda_status(convert_spinor(dst, dst_prec, src, src_prec, make_geom(dims),
                                    parity == WD_FULL ? 2 : 1, state().stream));
}

int wd_dslash_ex(void* out, const void* in, const void* gauge, int parity, int dagger, double a,
                 const void* x, double bx, const void* y, double cy, double* norm2,
                 const int dims[4], int prec, int recon) {
  const int tg = (recon & WD_TEMPORAL_GAUGE_BIT) != 0;
  const int staged = (recon & WD_STAGE_NEIGHBOURS) != 0;
  recon &= ~(WD_TEMPORAL_GAUGE_BIT | WD_STAGE_NEIGHBOURS);
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!out || !in || !gauge) return WD_ERR_NULL;
  if (!aligned(out) || !aligned(in) || !aligned(gauge) || (x && !aligned(x)) ||
      (y && !aligned(y)) || (norm2 && ((uintptr_t)norm2 & 7u)))
    return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD) return WD_ERR_ARG;
  if (link_bytes(prec, recon) == 0) return WD_ERR_PREC;
  if (out == in) return WD_ERR_ALIAS;
  Geom g = make_geom(dims);
  if (norm2) {
    cudaError_t e = ensure_scratch((size_t)((g.Vh + DSLASH_BS - 1) / DSLASH_BS) * 2);
    if (e != cudaSuccess) return cuda_status(e);
  }
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
  d.rs = scratch();
  d.g = g;
  d.parity = parity;
  d.tg = tg;
  if (staged) {
    if (prec != WD_F16 || recon != 12 || tg || norm2 || (g.S2 & 31) != 0) return WD_ERR_ARG;
    return cuda_status(launch_dslash_f16_staged(d, recon, dagger != 0, state().wait_limit,
                                                state().stream));
  }
  return cuda_status(launch_dslash(prec, d, recon, dagger != 0, state().stream));
}

static int dslash_common(void* out, const void* in, const void* gauge, double kappa, int parity,
                         const int dims[4], int prec, int dagger) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!out || !in || !gauge) return WD_ERR_NULL;
  if (parity == WD_FULL) {
    if (out == in) return WD_ERR_ALIAS;
    size_t h = spinor_half_bytes(make_geom(dims), prec);
    char* o = (char*)out;
    const char* i = (const char*)in;
    // out_e = in_e - kappa H_eo in_o ; out_o = in_o - kappa H_oe in_e
    WD_TRY(wd_dslash_ex(o, i + h, gauge, WD_EVEN, dagger, -kappa, i, 1.0, nullptr, 0.0, nullptr,
                        dims, prec, 12));
    return wd_dslash_ex(o + h, i, gauge, WD_ODD, dagger, -kappa, i + h, 1.0, nullptr, 0.0, nullptr,
                        dims, prec, 12);
  }
  return wd_dslash_ex(out, in, gauge, parity, dagger, -kappa, nullptr, 0.0, nullptr, 0.0, nullptr,
                      dims, prec, 12);
}

int wd_dslash(void* out, const void* in, const void* gauge, double kappa, int parity,
              const int dims[4], int prec) {
  return dslash_common(out, in, gauge, kappa, parity, dims, prec, 0);
}

int wd_dslash_dag(void* out, const void* in, const void* gauge, double kappa, int parity,
                  const int dims[4], int prec) {
  return dslash_common(out, in, gauge, kappa, parity, dims, prec, 1);
}

int wd_mhat(void* out, const void* in, const void* gauge, void* tmp, double kappa, int dagger,
            const int dims[4], int prec, int recon) {
  if (!tmp) return WD_ERR_NULL;
  if (tmp == in || tmp == out) return WD_ERR_ALIAS;
  WD_TRY(wd_dslash_ex(tmp, in, gauge, WD_ODD, dagger, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr,
                      dims, prec, recon));
  return wd_dslash_ex(out, tmp, gauge, WD_EVEN, dagger, -kappa * kappa, in, 1.0, nullptr, 0.0,
                      nullptr, dims, prec, recon);
}

int wd_dslash_mrhs(void* out, const void* in, const void* gauge, int parity, int dagger, double a,
                   const void* x, double bx, int nrhs, double* norm2, const int dims[4], int prec,
                   int recon) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!out || !in || !gauge) return WD_ERR_NULL;
  if (!aligned(out) || !aligned(in) || !aligned(gauge) || (x && !aligned(x)) ||
      (norm2 && ((uintptr_t)norm2 & 7u)))
    return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD) return WD_ERR_ARG;
  if (nrhs < 1 || nrhs > 32) return WD_ERR_ARG;
  if (link_bytes(prec, recon) == 0) return WD_ERR_PREC;
  if (out == in) return WD_ERR_ALIAS;
  return guarded([&] {
    return cuda_status(dslash_mrhs(out, in, gauge, parity, dagger, a, x, bx, nrhs, norm2,
                                   make_geom(dims), prec, recon, state().stream));
  });
}

int wd_set_autotune(int enable) { return set_autotune(enable); }

int wd_set_batch_mode(int mode) {
  if (mode != 0 && mode != 1) return -WD_ERR_ARG;
  return set_batch_mode(mode);
}

int wd_mrhs_set_lanes(int lanes) { return mrhs_set_lanes(lanes); }

int wd_dslash_set_block(int sites) { return dslash_set_block(sites); }

int wd_set_launch_overlap(int enable) { return set_launch_overlap(enable); }

int wd_tune_report(char* buf, size_t len) {
  return guarded([&] { return tune_report(buf, len); });
}

int wd_solve_batch(const wd_batch_problem* problems, int nproblems, const wd_solve_params* params,
                   wd_solve_info* info) {
  if (!problems) return WD_ERR_NULL;
  if (nproblems < 1 || nproblems > 16) return WD_ERR_ARG;
  for (int j = 0; j < nproblems; j++) {
    WD_TRY(check_dims(problems[j].dims));
    if (!problems[j].gauge || !problems[j].b || !problems[j].x) return WD_ERR_NULL;
    if (!aligned(problems[j].gauge) || !aligned(problems[j].b) || !aligned(problems[j].x))
      return WD_ERR_ALIGN;
    if (problems[j].nrhs < 1 || problems[j].nrhs > 32) return WD_ERR_ARG;
    if ((const void*)problems[j].x == (const void*)problems[j].b) return WD_ERR_ALIAS;
  }
  return guarded([&] { return solve_batch_impl(problems, nproblems, params, info); });
}

int wd_gauge_fix_temporal(double* U_out, double* omega_out, const double* U_in,
                          const int dims[4]) {
  WD_TRY(check_dims(dims));
  if (!U_out || !omega_out || !U_in) return WD_ERR_NULL;
  if (!aligned(U_out) || !aligned(omega_out) || !aligned(U_in)) return WD_ERR_ALIGN;
  if ((const void*)U_out == (const void*)U_in) return WD_ERR_ALIAS;
  return cuda_status(gauge_fix_temporal(U_out, omega_out, U_in, make_geom(dims), state().stream));
}

int wd_rotate_spinor(double* out, const double* in, const double* omega, const int dims[4],
                     int dagger) {
  WD_TRY(check_dims(dims));
  if (!out || !in || !omega) return WD_ERR_NULL;
  if (!aligned(out) || !aligned(in) || !aligned(omega)) return WD_ERR_ALIGN;
  return cuda_status(rotate_spinor(out, in, omega, make_geom(dims), dagger != 0, state().stream));
}

int wd_tc_gemm_bf16(float* D, const void* A, const void* B, int M, int K, int N) {
  if (!D || !A || !B) return WD_ERR_NULL;
  if (!aligned(D) || !aligned(A) || !aligned(B)) return WD_ERR_ALIGN;
  if (M < 128 || M % 128 || K < 16 || K % 16 || K > 256 || N < 16 || N % 16 || N > 256)
    return WD_ERR_ARG;
  cudaStream_t st = state().stream;
  int* flag = nullptr;
  WD_TRY(cuda_status(device_flag(&flag, st)));
  WD_TRY(cuda_status(tc_gemm_bf16(A, B, D, M, K, N, flag, st)));
  int h = 0;
  WD_TRY(cuda_status(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st)));
  WD_TRY(cuda_status(cudaStreamSynchronize(st)));
  return h ? WD_ERR_TIMEOUT : WD_OK;
}

int wd_set_wait_limit(long long polls) {
  if (polls < 0 || polls > (1LL << 26)) return WD_ERR_ARG;
  state().wait_limit = (long)polls;
  return WD_OK;
}

int wd_async_status(void) {
  int fault = 0;
  WD_TRY(cuda_status(stage_fault_take(&fault, state().stream)));
  return fault ? WD_ERR_TIMEOUT : WD_OK;
}

int wd_wait_selftest(long long spins) {
  if (spins < 1 || spins > (1LL << 24)) return WD_ERR_ARG;
  cudaStream_t st = state().stream;
  int* flag = nullptr;
  WD_TRY(cuda_status(device_flag(&flag, st)));
  WD_TRY(cuda_status(wait_selftest((long)spins, flag, st)));
  int h = 0;
  WD_TRY(cuda_status(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st)));
  WD_TRY(cuda_status(cudaStreamSynchronize(st)));
  return h ? WD_ERR_TIMEOUT : WD_OK;
}

void wd_nn_train_params_default(wd_nn_train_params* p) {
  if (!p) return;
  p->samples = 4096;
  p->batch = 16;
  p->epochs = 1;
  p->lr = 2e-3f;
  p->seed = 4242ull;
  p->init = 1;
  p->smooth = 0;
}

int wd_nn_layer(void* out, const void* in, const float* weights, int cin, int cout,
                const void* gauge, const int dims[4]) {
  WD_TRY(check_dims(dims));
  if (!out || !in || !weights || !gauge) return WD_ERR_NULL;
  if (!aligned(out) || !aligned(in) || !aligned(weights) || !aligned(gauge)) return WD_ERR_ALIGN;
  if ((cin != 4 && cin != 8) || (cout != 4 && cout != 8)) return WD_ERR_ARG;
  if (out == in) return WD_ERR_ALIAS;
  return guarded([&] { return nn_layer_impl(out, in, weights, cin, cout, gauge, dims); });
}

int wd_nn_wgrad(float* grad, const void* in, const void* delta, int cin, int cout,
                const void* gauge, const int dims[4]) {
  WD_TRY(check_dims(dims));
  if (!grad || !in || !delta || !gauge) return WD_ERR_NULL;
  if (!aligned(grad) || !aligned(in) || !aligned(delta) || !aligned(gauge)) return WD_ERR_ALIGN;
  if ((cin != 4 && cin != 8) || (cout != 4 && cout != 8) || (cin == 4 && cout == 4))
    return WD_ERR_ARG;
  return guarded([&] { return nn_wgrad_impl(grad, in, delta, cin, cout, gauge, dims); });
}

int wd_gaussian_spinor(void* out, unsigned long long seed, unsigned long long stream,
                       unsigned long long first, const int dims[4]) {
  WD_TRY(check_dims(dims));
  if (!out) return WD_ERR_NULL;
  if (!aligned(out)) return WD_ERR_ALIGN;
  return gaussian_spinor_impl(out, seed, stream, first, dims);
}

int wd_nn_init(float* weights, double kappa) {
  if (!weights) return WD_ERR_NULL;
  if (!aligned(weights)) return WD_ERR_ALIGN;
  return guarded([&] { return nn_init_impl(weights, kappa); });
}

int wd_nn_apply(void* out, const void* in, const float* weights, const void* gauge,
                const int dims[4]) {
  WD_TRY(check_dims(dims));
  if (!out || !in || !weights || !gauge) return WD_ERR_NULL;
  if (!aligned(out) || !aligned(in) || !aligned(weights) || !aligned(gauge)) return WD_ERR_ALIGN;
  if (out == in) return WD_ERR_ALIAS;
  return guarded([&] { return nn_apply_impl(out, in, weights, gauge, dims); });
}

int wd_nn_apply_ex(void* out, const void* in, const float* weights, const void* gauge,
                   const int dims[4], int flags) {
  WD_TRY(check_dims(dims));
  if (!out || !in || !weights || !gauge) return WD_ERR_NULL;
  if (!aligned(out) || !aligned(in) || !aligned(weights) || !aligned(gauge)) return WD_ERR_ALIGN;
  if (out == in) return WD_ERR_ALIAS;
  if (flags & ~(WD_NN_BF16 | WD_NN_EVEN)) return WD_ERR_ARG;
  return guarded([&] { return nn_apply_ex_impl(out, in, weights, gauge, dims, flags); });
}

int wd_nn_train(float* weights, const double* gauge, double kappa, const int dims[4],
                const wd_nn_train_params* params, wd_nn_train_info* info) {
  WD_TRY(check_dims(dims));
  if (!weights || !gauge) return WD_ERR_NULL;
  if (!aligned(weights) || !aligned(gauge)) return WD_ERR_ALIGN;
  wd_nn_train_params p;
  wd_nn_train_params_default(&p);
  if (params) p = *params;
  return guarded([&] { return nn_train_impl(weights, gauge, kappa, dims, &p, info); });
}

int wd_solve_fgcr(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
                  const float* weights, int m, const wd_solve_params* params,
                  wd_solve_info* info) {
  WD_TRY(check_dims(dims));
  if (!x || !b || !gauge) return WD_ERR_NULL;
  if (!aligned(x) || !aligned(b) || !aligned(gauge) || (weights && !aligned(weights)))
    return WD_ERR_ALIGN;
  if (x == b) return WD_ERR_ALIAS;
  if (m < 1 || m > 16) return WD_ERR_ARG;
  return guarded([&] { return fgcr_impl(x, b, gauge, kappa, dims, weights, params, info, m); });
}

int wd_solve_fcg(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
                 const float* weights, const wd_solve_params* params, wd_solve_info* info) {
  WD_TRY(check_dims(dims));
  if (!x || !b || !gauge) return WD_ERR_NULL;
  if (!aligned(x) || !aligned(b) || !aligned(gauge) || (weights && !aligned(weights)))
    return WD_ERR_ALIGN;
  if (x == b) return WD_ERR_ALIAS;
  return guarded([&] { return fcg_impl(x, b, gauge, kappa, dims, weights, params, info); });
}

int wd_norm2(double* result, const void* x, const int dims[4], int parity, int prec) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!result || !x) return WD_ERR_NULL;
  if (!aligned(x) || ((uintptr_t)result & 7u)) return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return WD_ERR_ARG;
  return cuda_status(norm2(result, x, make_geom(dims), prec, parity == WD_FULL ? 2 : 1,
                           state().stream));
}

int wd_cdot(double* result, const void* x, const void* y, const int dims[4], int parity,
            int prec) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!result || !x || !y) return WD_ERR_NULL;
  if (!aligned(x) || !aligned(y) || ((uintptr_t)result & 7u)) return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return WD_ERR_ARG;
  return cuda_status(cdot(result, x, y, make_geom(dims), prec, parity == WD_FULL ? 2 : 1,
                          state().stream));
}

int wd_axpby(double a, const void* x, double b, void* y, const int dims[4], int parity, int prec) {
  WD_TRY(check_dims(dims));
  WD_TRY(check_prec(prec));
  if (!x || !y) return WD_ERR_NULL;
  if (!aligned(x) || !aligned(y)) return WD_ERR_ALIGN;
  if (parity != WD_EVEN && parity != WD_ODD && parity != WD_FULL) return WD_ERR_ARG;
  return cuda_status(axpby(a, x, b, y, make_geom(dims), prec, parity == WD_FULL ? 2 : 1,
                           state().stream));
}

void wd_solve_params_default(wd_solve_params* p) {
  if (!p) return;
  p->inner_prec = WD_F32;
  p->inner_recon = 12;
  p->outer_recon = 18;
  p->reliable_interval = 50;
  p->check_interval = 10;
  p->maxiter = 100000;
  p->use_graph = 1;
  p->use_initial_guess = 0;
  p->tol = 1e-10;
  p->gauge_fix = 0;
  p->solver = WD_SOLVER_CG;
}

int wd_solve_ex(double* x, const double* b, const double* gauge, double kappa, const int dims[4],
                const wd_solve_params* params, wd_solve_info* info) {
  WD_TRY(check_dims(dims));
  if (!x || !b || !gauge) return WD_ERR_NULL;
  if (!aligned(x) || !aligned(b) || !aligned(gauge)) return WD_ERR_ALIGN;
  if (x == b) return WD_ERR_ALIAS;
  return solve_impl(x, b, gauge, kappa, dims, params, info);
}

int wd_solve(double* x, const double* b, const double* gauge, double kappa, double tol,
             const int dims[4]) {
  wd_solve_params p;
  wd_solve_params_default(&p);
  p.tol = tol;
  return wd_solve_ex(x, b, gauge, kappa, dims, &p, nullptr);
}

}  // extern "C"
