// Diagnostics of a cavity state (Punia & Ray, arXiv:2411.06563, Sec. 4.2-4.3): local Nusselt
// number on the hot and cold walls, Nu_avg(z) = (1/Ly) int_0^Ly Nu_local dy, its maximum over z,
// wall means (over the wall area Ly Lz), the entropy-generation fields E_HT = |grad theta|^2,
// E_FF = phi eta I2 (chi* = phi* = phi), E_local = E_HT + E_FF, their integrals over the box and
// the Bejan number E_HT / E_total. Integrals use composite Simpson weights with the spacing of
// each direction (N odd; trapezoid for even N); all in double.

#include <math.h>

#include "hosc_device.cuh"
#include "hosc_internal.h"

namespace hosc {

namespace {

__device__ __forceinline__ double simpson_w(int a, int N, double h) {
  if (N % 2 == 1) {
    if (a == 0 || a == N - 1) return h / 3.0;
    return (a % 2 == 1) ? 4.0 * h / 3.0 : 2.0 * h / 3.0;
  }
  return (a == 0 || a == N - 1) ? 0.5 * h : h;
}

// Nu_local(y, z) = -d theta/dx at x = 0 (fourth-order one-sided), and -d theta/dx at x = 1.
__global__ void k_nu_local(DevParams P, const double* __restrict__ th, double* nu_hot,
                           double* nu_cold) {
  const int N = P.N;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)N * N) return;
  const int j = (int)(t % N), k = (int)(t / N);
  const long c0 = node(0, j, k, N), c1 = node(N - 1, j, k, N);
  const double inv = 1.0 / (12.0 * P.h);
  const double d0 = (-25.0 * th[c0] + 48.0 * th[c0 + 1] - 36.0 * th[c0 + 2] + 16.0 * th[c0 + 3] -
                     3.0 * th[c0 + 4]) * inv;
  const double d1 = (25.0 * th[c1] - 48.0 * th[c1 - 1] + 36.0 * th[c1 - 2] - 16.0 * th[c1 - 3] +
                     3.0 * th[c1 - 4]) * inv;
  nu_hot[t] = -d0;
  nu_cold[t] = -d1;
}

// One block: Nu_avg(z) (Simpson in y), its maximum, and the Simpson surface means.
__global__ void k_nu_reduce(DevParams P, const double* nu_hot, const double* nu_cold,
                            double* nu_avg, double* scal) {
  __shared__ double smem[32 * 2];
  const int N = P.N;
  const double hy = P.Ly / (N - 1), hz = P.Lz / (N - 1);
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += nu_hot[j + (long)N * k] * simpson_w(j, N, hy);
    nu_avg[k] = s;   // divided by Ly below, after the surface sums
  }
  __syncthreads();
  double acc[2] = {0.0, 0.0};
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    double sc = 0.0;
    for (int j = 0; j < N; ++j) sc += nu_cold[j + (long)N * k] * simpson_w(j, N, hy);
    acc[0] += simpson_w(k, N, hz) * nu_avg[k];
    acc[1] += simpson_w(k, N, hz) * sc;
  }
  block_reduce<2, false>(acc, smem);
  __syncthreads();   // every nu_avg read above precedes its scaling
  for (int k = threadIdx.x; k < N; k += blockDim.x) nu_avg[k] /= P.Ly;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = -INFINITY;
    for (int k = 0; k < N; ++k) mx = fmax(mx, nu_avg[k]);
    const double area = P.Ly * P.Lz;
    scal[0] = mx;
    scal[1] = acc[0] / area;
    scal[2] = acc[1] / area;
  }
}

// E_HT, E_FF, E_local at every node (optionally stored) and their Simpson volume integrals.
__global__ void __launch_bounds__(kThreads) k_entropy(DevParams P, const double* __restrict__ u,
                                                     const double* __restrict__ v,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ th, double* eloc,
                                                     int store, double* red,
                                                     unsigned int* counter, int nblocks,
                                                     double* scal) {
  __shared__ double smem[32 * 2];
  const int N = P.N;
  const long n3 = (long)N * N * N;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (t < n3) {
    const int i = (int)(t % N), j = (int)((t / N) % N), k = (int)(t / ((long)N * N));
    const double ix = P.inv2[0], iy = P.inv2[1], iz = P.inv2[2];
    const double tx = grad_axis(th, t, i, N, 1, ix);
    const double ty = grad_axis(th, t, j, N, N, iy);
    const double tz = grad_axis(th, t, k, N, (long)N * N, iz);
    const double eht = tx * tx + ty * ty + tz * tz;
    const Grad9 g = velocity_gradients(u, v, w, i, j, k, N, ix, iy, iz);
    const double I2 = second_invariant(g);
    double eta = 1.0;
    if (!P.newtonian) {
      // the viscosity of S1, including its edge and corner rule
      const int wi = (i == 0) | (i == N - 1), wj = (j == 0) | (j == N - 1),
                wk = (k == 0) | (k == N - 1);
      int a = i, b = j, cc = k;
      if (wi + wj + wk >= 2) {
        a = (i == 0) ? 1 : (i == N - 1 ? N - 2 : i);
        b = (j == 0) ? 1 : (j == N - 1 ? N - 2 : j);
        cc = (k == 0) ? 1 : (k == N - 1 ? N - 2 : k);
      }
      const Grad9 ge = velocity_gradients(u, v, w, a, b, cc, N, ix, iy, iz);
      eta = pow(second_invariant(ge) + P.I2_eps, 0.5 * (P.n - 1.0));
    }
    const double eff = P.phi * eta * I2;
    if (store) {
      eloc[t] = eht;
      eloc[n3 + t] = eff;
      eloc[2 * n3 + t] = eht + eff;
    }
    const double wgt = simpson_w(i, N, P.h) * simpson_w(j, N, P.Ly / (N - 1)) *
                       simpson_w(k, N, P.Lz / (N - 1));
    acc[0] = wgt * eht;
    acc[1] = wgt * eff;
  }
  block_reduce<2, false>(acc, smem);
  if (publish_is_last<2>(acc, red, counter)) {
    double tot[2];
    reduce_partials<2, false>(tot, red, nblocks, counter, smem);
    if (threadIdx.x == 0) {
      scal[3] = tot[0];
      scal[4] = tot[1];
    }
  }
}

}  // namespace

void launch_diagnostics(const DevParams& P, const Fields& F, int cur, int want_fields,
                        cudaStream_t s) {
  const long N = P.N, n3 = N * N * N;
  k_nu_local<<<red_blocks(N * N), kThreads, 0, s>>>(P, F.th, F.nu_hot, F.nu_cold);
  k_nu_reduce<<<1, kThreads, 0, s>>>(P, F.nu_hot, F.nu_cold, F.nu_avg, F.diag_scal);
  const int b = red_blocks(n3);
  k_entropy<<<b, kThreads, 0, s>>>(P, F.u[cur], F.v[cur], F.w[cur], F.th, F.eloc, want_fields,
                                   F.red, F.counter, b, F.diag_scal);
}

}  // namespace hosc
