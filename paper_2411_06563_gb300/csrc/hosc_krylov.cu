// Unpreconditioned BiCGSTAB (van der Vorst) on the four HOSC systems of one step (Punia & Ray,
// arXiv:2411.06563, Sec. 2.2: the implicit seven-point systems are solved with BiCGSTAB without
// preconditioning).
//
// The four systems (u, v, w with the shared momentum operator, theta with the energy operator)
// advance together, each with its own scalars. The operator is applied matrix-free from the seven
// weights per node written by the right-hand-side kernel. Unknown is the increment
// x = chi^{n+1} - chi^n, zero on the walls, started at x = 0, so r_0 = dt (R - B chi^n); the
// shadow residual is r_0 (kept in rhs[]). Stop when ||r_k||_2 <= tol ||r_0||_2.
//
// One iteration = three kernels; each ends with a last-block reduction that finalises the scalar
// the next kernel needs (alpha, omega, beta / convergence). No kernel waits on another block.

#include <math.h>

#include "hosc_device.cuh"
#include "hosc_internal.h"

namespace hosc {

namespace {

__device__ __forceinline__ double apply7(const double* const* A, long c, double x0, double xp,
                                         double xm, double yp, double ym, double zp, double zm) {
  return A[0][c] * x0 + A[1][c] * xp + A[2][c] * xm + A[3][c] * yp + A[4][c] * ym +
         A[5][c] * zp + A[6][c] * zm;
}

__device__ __forceinline__ bool interior_index(const DevParams& P, long t, long& c) {
  const int N = P.N, ni = N - 2;
  const long cnt = (long)ni * ni * ni;
  if (t >= cnt) return false;
  const int i = 1 + (int)(t % ni), j = 1 + (int)((t / ni) % ni), k = 1 + (int)(t / ((long)ni * ni));
  c = node(i, j, k, N);
  return true;
}

// Algorithmic bytes of one launch: every array element the active systems touch, once.
__device__ __forceinline__ double launch_bytes(const DevParams& P, const int done[4],
                                               double per_system_words, double coeff_words) {
  const double ni = (double)(P.N - 2);
  const int nm = !done[0] + !done[1] + !done[2], ne = !done[3];
  const double words = per_system_words * (nm + ne) + coeff_words * ((nm > 0) + ne);
  return 8.0 * ni * ni * ni * words;
}

// r = r_0 = rhs, x = 0, p = v = 0; ||r_0||^2 per system.
__global__ void __launch_bounds__(kThreads) k_bicg_init(DevParams P, Fields F, int nblocks) {
  __shared__ double smem[32 * 4];
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long c;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (interior_index(P, t, c)) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const double r = F.rhs[s][c];
      F.r[s][c] = r;
      F.x[s][c] = 0.0;
      F.pk[0][s][c] = 0.0;
      F.pk[1][s][c] = 0.0;
      F.vk[0][s][c] = 0.0;
      F.vk[1][s][c] = 0.0;
      acc[s] = r * r;
    }
  }
  block_reduce<4, false>(acc, smem);
  if (publish_is_last<4>(acc, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        k.r0norm = sqrt(tot[s]);
        k.rnorm = k.r0norm;
        k.rho = tot[s];
        k.alpha = 1.0;
        k.omega = 1.0;
        k.beta = 0.0;
        k.iters = 0;
        k.status = 0;
        k.done = (k.r0norm == 0.0) ? 1 : 0;
      }
    }
  }
}

// p_new = r + beta (p_old - omega v_old) on the fly at the 7 stencil nodes, v_new = A p_new,
// partial r0 . v_new; last block: alpha = rho / (r0 . v).
__global__ void __launch_bounds__(kThreads) k_bicg_pv(DevParams P, Fields F, int pp, int nblocks) {
  __shared__ double smem[32 * 4];
  __shared__ double s_beta[4], s_omega[4];
  __shared__ int s_done[4];
  if (threadIdx.x < 4) {
    s_beta[threadIdx.x] = F.ks[threadIdx.x].beta;
    s_omega[threadIdx.x] = F.ks[threadIdx.x].omega;
    s_done[threadIdx.x] = F.ks[threadIdx.x].done;
  }
  __syncthreads();
  if (s_done[0] & s_done[1] & s_done[2] & s_done[3]) return;  // uniform over the grid
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long sy = P.N, sz = (long)P.N * P.N;
  long c;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (interior_index(P, t, c)) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (s_done[s]) continue;
      const double* r = F.r[s];
      const double* po = F.pk[pp][s];
      const double* vo = F.vk[pp][s];
      const double b = s_beta[s], om = s_omega[s];
      const long nb[7] = {c, c + 1, c - 1, c + sy, c - sy, c + sz, c - sz};
      double pn[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) pn[q] = r[nb[q]] + b * (po[nb[q]] - om * vo[nb[q]]);
      const double* const* A = (s < 3) ? F.Am : F.Ae;
      const double vn = apply7(A, c, pn[0], pn[1], pn[2], pn[3], pn[4], pn[5], pn[6]);
      F.pk[1 - pp][s][c] = pn[0];
      F.vk[1 - pp][s][c] = vn;
      acc[s] = F.rhs[s][c] * vn;
    }
  }
  block_reduce<4, false>(acc, smem);
  if (publish_is_last<4>(acc, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        if (tot[s] == 0.0 || !isfinite(tot[s])) {
          k.done = 1;
          k.status = HOSC_ENOCONV;
          continue;
        }
        k.alpha = k.rho / tot[s];
      }
      F.alg_bytes[HOSC_K_BICG_PV] += launch_bytes(P, s_done, 6.0, 7.0);
    }
  }
}

// s = r - alpha v on the fly at the 7 stencil nodes, t = A s, partials (t . s, t . t);
// last block: omega = (t . s)/(t . t) (0 when t = 0).
__global__ void __launch_bounds__(kThreads) k_bicg_st(DevParams P, Fields F, int pp, int nblocks) {
  __shared__ double smem[32 * 8];
  __shared__ double s_alpha[4];
  __shared__ int s_done[4];
  if (threadIdx.x < 4) {
    s_alpha[threadIdx.x] = F.ks[threadIdx.x].alpha;
    s_done[threadIdx.x] = F.ks[threadIdx.x].done;
  }
  __syncthreads();
  if (s_done[0] & s_done[1] & s_done[2] & s_done[3]) return;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long sy = P.N, sz = (long)P.N * P.N;
  const int np = 1 - pp;   // buffers written by k_bicg_pv of this iteration
  long c;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (interior_index(P, t, c)) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (s_done[s]) continue;
      const double* r = F.r[s];
      const double* v = F.vk[np][s];
      const double a = s_alpha[s];
      const long nb[7] = {c, c + 1, c - 1, c + sy, c - sy, c + sz, c - sz};
      double sv[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) sv[q] = r[nb[q]] - a * v[nb[q]];
      const double* const* A = (s < 3) ? F.Am : F.Ae;
      const double tv = apply7(A, c, sv[0], sv[1], sv[2], sv[3], sv[4], sv[5], sv[6]);
      F.t[s][c] = tv;
      acc[2 * s] = tv * sv[0];
      acc[2 * s + 1] = tv * tv;
    }
  }
  block_reduce<8, false>(acc, smem);
  if (publish_is_last<8>(acc, F.red, F.counter)) {
    double tot[8];
    reduce_partials<8, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        k.omega = tot[2 * s + 1] > 0.0 ? tot[2 * s] / tot[2 * s + 1] : 0.0;
      }
      F.alg_bytes[HOSC_K_BICG_ST] += launch_bytes(P, s_done, 3.0, 7.0);
    }
  }
}

// s = r - alpha v; x += alpha p + omega s; r = s - omega t; partials (r0 . r, r . r);
// last block: convergence test, breakdown test, beta and rho for the next iteration.
__global__ void __launch_bounds__(kThreads) k_bicg_xr(DevParams P, Fields F, int pp, int nblocks) {
  __shared__ double smem[32 * 8];
  __shared__ double s_alpha[4], s_omega[4];
  __shared__ int s_done[4];
  if (threadIdx.x < 4) {
    s_alpha[threadIdx.x] = F.ks[threadIdx.x].alpha;
    s_omega[threadIdx.x] = F.ks[threadIdx.x].omega;
    s_done[threadIdx.x] = F.ks[threadIdx.x].done;
  }
  __syncthreads();
  if (s_done[0] & s_done[1] & s_done[2] & s_done[3]) return;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = 1 - pp;
  long c;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (interior_index(P, t, c)) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (s_done[s]) continue;
      const double a = s_alpha[s], om = s_omega[s];
      const double sv = F.r[s][c] - a * F.vk[np][s][c];
      F.x[s][c] = F.x[s][c] + a * F.pk[np][s][c] + om * sv;
      const double rn = sv - om * F.t[s][c];
      F.r[s][c] = rn;
      acc[2 * s] = F.rhs[s][c] * rn;
      acc[2 * s + 1] = rn * rn;
    }
  }
  block_reduce<8, false>(acc, smem);
  if (publish_is_last<8>(acc, F.red, F.counter)) {
    double tot[8];
    reduce_partials<8, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        const double rho_new = tot[2 * s];
        k.rnorm = sqrt(tot[2 * s + 1]);
        k.iters += 1;
        if (k.rnorm <= P.tol_lin * k.r0norm) {
          k.done = 1;
          k.status = 0;
        } else if (!isfinite(k.rnorm) || k.iters >= P.max_lin_iter || rho_new == 0.0 ||
                   k.omega == 0.0) {
          k.done = 1;
          k.status = HOSC_ENOCONV;
        } else {
          k.beta = (rho_new / k.rho) * (k.alpha / k.omega);
          k.rho = rho_new;
        }
      }
      F.alg_bytes[HOSC_K_BICG_XR] += launch_bytes(P, s_done, 8.0, 0.0);
    }
  }
}

int interior_blocks(const DevParams& P) {
  const long ni = P.N - 2;
  return red_blocks(ni * ni * ni);
}

}  // namespace

void launch_bicg_init(const DevParams& P, const Fields& F, cudaStream_t s) {
  const int b = interior_blocks(P);
  k_bicg_init<<<b, kThreads, 0, s>>>(P, F, b);
}

void launch_bicg_pv(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  const int b = interior_blocks(P);
  k_bicg_pv<<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_bicg_st(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  const int b = interior_blocks(P);
  k_bicg_st<<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_bicg_xr(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  const int b = interior_blocks(P);
  k_bicg_xr<<<b, kThreads, 0, s>>>(P, F, pp, b);
}

}  // namespace hosc
