// Temporal gauge fixing (the paper's gauge-fixing variant, section
// "Performance": the temporal links are fixed to the identity on all but one
// time slice, which saves their memory traffic in the hopping term).
//
// With Omega(x, t=0) = 1 and Omega(x, t+1) = Omega(x, t) U_t(x, t), the
// transformed links U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^+ have
// U'_t(x, t) = 1 for t < L3-1, while U'_t(x, L3-1) is the product of the time
// links along the line (the Polyakov loop).  The Wilson operator is gauge
// covariant, D[U'] = Omega D[U] Omega^+, so D[U] x = b is solved as
// D[U'] x' = Omega b with x = Omega^+ x'.
#include "wd_internal.h"

namespace wd {

__device__ __forceinline__ void mat_mul(cx<double> (&c)[9], const cx<double> (&a)[9],
                                        const cx<double> (&b)[9]) {
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cx<double> s = mk<double>(0, 0);
#pragma unroll
      for (int k = 0; k < 3; k++) s = cmadd(a[i * 3 + k], b[k * 3 + j], s);
      c[i * 3 + j] = s;
    }
}

// c = a b^+
__device__ __forceinline__ void mat_mul_dag(cx<double> (&c)[9], const cx<double> (&a)[9],
                                            const cx<double> (&b)[9]) {
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cx<double> s = mk<double>(0, 0);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        cx<double> bj = mk<double>(b[j * 3 + k].r, -b[j * 3 + k].i);
        s = cmadd(a[i * 3 + k], bj, s);
      }
      c[i * 3 + j] = s;
    }
}

__device__ __forceinline__ void ld9(cx<double> (&m)[9], const double2* p) {
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 v = p[k];
    m[k] = mk<double>(v.x, v.y);
  }
}

__device__ __forceinline__ void st9(double2* p, const cx<double> (&m)[9]) {
#pragma unroll
  for (int k = 0; k < 9; k++) p[k] = make_double2(m[k].r, m[k].i);
}

// one thread per spatial site: walk the time line
__global__ void temporal_omega_kernel(double2* omega, const double2* __restrict__ U, Geom g,
                                      long long S) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= S) return;
  const long long V = 2LL * g.Vh;
  cx<double> om[9];
#pragma unroll
  for (int k = 0; k < 9; k++) om[k] = mk<double>((k % 4) == 0 ? 1.0 : 0.0, 0.0);
  st9(omega + s * 9, om);
  for (int t = 0; t + 1 < g.L[3]; t++) {
    const long long i = s + S * t;
    cx<double> u[9], nx[9];
    ld9(u, U + (3 * V + i) * 9);
    mat_mul(nx, om, u);
#pragma unroll
    for (int k = 0; k < 9; k++) om[k] = nx[k];
    st9(omega + (i + S) * 9, om);
  }
}

// one thread per (mu, site): U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^+
__global__ void rotate_links_kernel(double2* Uout, const double2* __restrict__ Uin,
                                    const double2* __restrict__ omega, Geom g) {
  const long long V = 2LL * g.Vh;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 4 * V;
       t += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(t / V);
    const long long i = t - mu * V;
    int x[4];
    long long r = i;
    for (int m = 0; m < 4; m++) {
      x[m] = (int)(r % g.L[m]);
      r /= g.L[m];
    }
    cx<double> out[9];
    if (mu == 3 && x[3] < g.L[3] - 1) {
#pragma unroll
      for (int k = 0; k < 9; k++) out[k] = mk<double>((k % 4) == 0 ? 1.0 : 0.0, 0.0);
    } else {
      int y[4] = {x[0], x[1], x[2], x[3]};
      y[mu] = (y[mu] + 1) % g.L[mu];
      const long long j = y[0] + (long long)g.L[0] * (y[1] + (long long)g.L[1] * (y[2] + (long long)g.L[2] * y[3]));
      cx<double> a[9], u[9], b[9], tmp[9];
      ld9(a, omega + i * 9);
      ld9(u, Uin + t * 9);
      ld9(b, omega + j * 9);
      mat_mul(tmp, a, u);
      mat_mul_dag(out, tmp, b);
    }
    st9(Uout + t * 9, out);
  }
}

// out(x) = Omega(x) in(x)  (dagger: Omega(x)^+ in(x)), canonical full spinors
__global__ void rotate_spinor_kernel(double2* out, const double2* in,
                                     const double2* __restrict__ omega, Geom g, int dagger) {
  const long long V = 2LL * g.Vh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x) {
    cx<double> om[9], v[12], w[12];
    ld9(om, omega + i * 9);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 q = in[i * 12 + k];
      v[k] = mk<double>(q.x, q.y);
    }
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int a = 0; a < 3; a++) {
        cx<double> acc = mk<double>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; b++) {
          if (dagger)
            acc = cjmadd(om[b * 3 + a], v[s * 3 + b], acc);
          else
            acc = cmadd(om[a * 3 + b], v[s * 3 + b], acc);
        }
        w[s * 3 + a] = acc;
      }
#pragma unroll
    for (int k = 0; k < 12; k++) out[i * 12 + k] = make_double2(w[k].r, w[k].i);
  }
}

cudaError_t gauge_fix_temporal(double* Uout, double* omega, const double* Uin, const Geom& g,
                               cudaStream_t st) {
  const long long S = (long long)g.L[0] * g.L[1] * g.L[2];
  temporal_omega_kernel<<<(unsigned)((S + 127) / 128), 128, 0, st>>>((double2*)omega,
                                                                     (const double2*)Uin, g, S);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rotate_links_kernel<<<blas_grid(8LL * g.Vh, 256), 256, 0, st>>>(
      (double2*)Uout, (const double2*)Uin, (const double2*)omega, g);
  return cudaGetLastError();
}

cudaError_t rotate_spinor(double* out, const double* in, const double* omega, const Geom& g,
                          int dagger, cudaStream_t st) {
  rotate_spinor_kernel<<<blas_grid(2LL * g.Vh, 256), 256, 0, st>>>(
      (double2*)out, (const double2*)in, (const double2*)omega, g, dagger);
  return cudaGetLastError();
}

}  // namespace wd
