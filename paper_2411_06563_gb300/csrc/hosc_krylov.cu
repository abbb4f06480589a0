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
//
// Two storage forms. FP64 (planar): one array per system and per weight, one thread per interior
// node. Mixed precision (interleaved, float): one float4 per node holds the four systems, the
// fourteen weights sit in four float4 per node, and a thread owns one interior (i, j) column over
// a segment of kz planes, keeping the z-neighbours in registers as it marches; its dot-product
// terms accumulate in float-float over the segment before the block reduction.

#include <math.h>

#include "hosc_device.cuh"
#include "hosc_internal.h"
#include "hosc_krylov4.cuh"

namespace hosc {

namespace {

template <class T>
__device__ __forceinline__ T apply7(const T* const* A, int c, T x0, T xp, T xm, T yp, T ym, T zp,
                                    T zm) {
  return A[0][c] * x0 + A[1][c] * xp + A[2][c] * xm + A[3][c] * yp + A[4][c] * ym +
         A[5][c] * zp + A[6][c] * zm;
}

template <class T>
__device__ __forceinline__ T* vec(double* p) { return reinterpret_cast<T*>(p); }
template <class T>
__device__ __forceinline__ const T* const* ops(double* const* p) {
  return reinterpret_cast<const T* const*>(p);
}

// Thread t -> interior node (1 + t % ni, ...) in 32-bit arithmetic (N^3 < 2^31 for N <= 1025).
// Thread t -> interior node (1 + t % ni, ...) in 32-bit arithmetic (N^3 < 2^31 for N <= 1025).
__device__ __forceinline__ bool interior_index(const DevParams& P, unsigned t, int& c) {
  const unsigned N = P.N, ni = N - 2;
  if (t >= ni * ni * ni) return false;
  const unsigned q = t / ni;
  const unsigned i = t - q * ni, j = q % ni, k = q / ni;
  c = (int)((i + 1) + N * ((j + 1) + N * (k + 1)));
  return true;
}

// Algorithmic bytes of one launch: every array element the active systems touch, once.
__device__ __forceinline__ double launch_bytes(const DevParams& P, const int done[4],
                                               double per_system_words, double coeff_words,
                                               double word_bytes) {
  const double ni = (double)(P.N - 2);
  const int nm = !done[0] + !done[1] + !done[2], ne = !done[3];
  const double words = per_system_words * (nm + ne) + coeff_words * ((nm > 0) + ne);
  return word_bytes * ni * ni * ni * words;
}

// Block partial of M dot-product terms a[m] * b[m] in double (valid in thread 0).
template <int M>
__device__ __forceinline__ void block_partial(const double (&a)[M], const double (&b)[M],
                                              double (&out)[M], double* smem) {
#pragma unroll
  for (int m = 0; m < M; ++m) out[m] = a[m] * b[m];
  block_reduce<M, false>(out, smem);
}

// r = r_0 = rhs, x = 0, p = v = 0; ||r_0||^2 per system.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bicg_init(DevParams P, Fields F, int nblocks) {
  __shared__ double smem[32 * 4];
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  int c;
  T da[4] = {T(0), T(0), T(0), T(0)}, db[4] = {T(0), T(0), T(0), T(0)};
  if (interior_index(P, t, c)) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const T r = vec<T>(F.rhs[s])[c];
      vec<T>(F.r[s])[c] = r;
      vec<T>(F.x[s])[c] = T(0);
      vec<T>(F.pk[0][s])[c] = T(0);
      vec<T>(F.pk[1][s])[c] = T(0);
      vec<T>(F.vk[0][s])[c] = T(0);
      vec<T>(F.vk[1][s])[c] = T(0);
      if (P.solver == 1) vec<T>(F.u0[s])[c] = T(0);
      da[s] = r;
      db[s] = r;
    }
  }
  double part[4];
  block_partial<4>(da, db, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        k.r0norm = sqrt(tot[s]);
        k.rnorm = k.r0norm;
        k.rho = tot[s];   // BiCGSTAB(2): rho_0 after the first cycle's rho_0 = -omega rho_0, j = 0
        k.alpha = P.solver == 1 ? 0.0 : 1.0;
        k.omega = 1.0;
        k.beta = 0.0;
        k.g1 = k.g2 = 0.0;
        k.iters = 0;
        k.status = 0;
        // an inner pressure pass solves the momentum systems only
        k.done = (k.r0norm == 0.0 || *F.halt || (s == 3 && P.inner_pass)) ? 1 : 0;
      }
    }
  }
}

// End of one pass of the captured BiCGSTAB loop body: continue while a system is iterating.
// Bounded: k_bicg_xr marks a system done at max_lin_iter at the latest.
__global__ void k_loop_cond(const KrylovScalars* ks, cudaGraphConditionalHandle handle) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const unsigned more = !(ks[0].done && ks[1].done && ks[2].done && ks[3].done);
    cudaGraphSetConditional(handle, more);
  }
}

// p_new = r + beta (p_old - omega v_old) on the fly at the 7 stencil nodes, v_new = A p_new,
// partial r0 . v_new; last block: alpha = rho / (r0 . v).
template <class T>
__global__ void __launch_bounds__(kThreads) k_bicg_pv(DevParams P, Fields F, int pp, int nblocks) {
  __shared__ double smem[32 * 4];
  __shared__ T s_beta[4], s_omega[4];
  __shared__ int s_done[4];
  if (threadIdx.x < 4) {
    s_beta[threadIdx.x] = (T)F.ks[threadIdx.x].beta;
    s_omega[threadIdx.x] = (T)F.ks[threadIdx.x].omega;
    s_done[threadIdx.x] = F.ks[threadIdx.x].done;
  }
  __syncthreads();
  if (s_done[0] & s_done[1] & s_done[2] & s_done[3]) return;  // uniform over the grid
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int sy = P.N, sz = P.N * P.N;
  int c;
  T da[4] = {T(0), T(0), T(0), T(0)}, db[4] = {T(0), T(0), T(0), T(0)};
  if (interior_index(P, t, c)) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (s_done[s]) continue;
      const T* r = vec<T>(F.r[s]);
      const T* po = vec<T>(F.pk[pp][s]);
      const T* vo = vec<T>(F.vk[pp][s]);
      const T b = s_beta[s], om = s_omega[s];
      const int nb[7] = {c, c + 1, c - 1, c + sy, c - sy, c + sz, c - sz};
      T pn[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) pn[q] = r[nb[q]] + b * (po[nb[q]] - om * vo[nb[q]]);
      const T* const* A = (s < 3) ? ops<T>(F.Am) : ops<T>(F.Ae);
      const T vn = apply7<T>(A, c, pn[0], pn[1], pn[2], pn[3], pn[4], pn[5], pn[6]);
      vec<T>(F.pk[1 - pp][s])[c] = pn[0];
      vec<T>(F.vk[1 - pp][s])[c] = vn;
      da[s] = vec<T>(F.rhs[s])[c];
      db[s] = vn;
    }
  }
  double part[4];
  block_partial<4>(da, db, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
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
      F.alg_bytes[HOSC_K_BICG_PV] += launch_bytes(P, s_done, 6.0, 7.0, sizeof(T));
    }
  }
}

// s = r - alpha v on the fly at the 7 stencil nodes, t = A s, partials (t . s, t . t);
// last block: omega = (t . s)/(t . t) (0 when t = 0).
template <class T>
__global__ void __launch_bounds__(kThreads) k_bicg_st(DevParams P, Fields F, int pp, int nblocks) {
  __shared__ double smem[32 * 8];
  __shared__ T s_alpha[4];
  __shared__ int s_done[4];
  if (threadIdx.x < 4) {
    s_alpha[threadIdx.x] = (T)F.ks[threadIdx.x].alpha;
    s_done[threadIdx.x] = F.ks[threadIdx.x].done;
  }
  __syncthreads();
  if (s_done[0] & s_done[1] & s_done[2] & s_done[3]) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int sy = P.N, sz = P.N * P.N;
  const int np = 1 - pp;   // buffers written by k_bicg_pv of this iteration
  int c;
  T da[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T db[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  if (interior_index(P, t, c)) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (s_done[s]) continue;
      const T* r = vec<T>(F.r[s]);
      const T* v = vec<T>(F.vk[np][s]);
      const T a = s_alpha[s];
      const int nb[7] = {c, c + 1, c - 1, c + sy, c - sy, c + sz, c - sz};
      T sv[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) sv[q] = r[nb[q]] - a * v[nb[q]];
      const T* const* A = (s < 3) ? ops<T>(F.Am) : ops<T>(F.Ae);
      const T tv = apply7<T>(A, c, sv[0], sv[1], sv[2], sv[3], sv[4], sv[5], sv[6]);
      vec<T>(F.t[s])[c] = tv;
      da[2 * s] = tv;
      db[2 * s] = sv[0];
      da[2 * s + 1] = tv;
      db[2 * s + 1] = tv;
    }
  }
  double part[8];
  block_partial<8>(da, db, part, smem);
  if (publish_is_last<8>(part, F.red, F.counter)) {
    double tot[8];
    reduce_partials<8, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        k.omega = tot[2 * s + 1] > 0.0 ? tot[2 * s] / tot[2 * s + 1] : 0.0;
      }
      F.alg_bytes[HOSC_K_BICG_ST] += launch_bytes(P, s_done, 3.0, 7.0, sizeof(T));
    }
  }
}

// s = r - alpha v; x += alpha p + omega s; r = s - omega t; partials (r0 . r, r . r);
// last block: convergence test, breakdown test, beta and rho for the next iteration.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bicg_xr(DevParams P, Fields F, int pp, int nblocks) {
  __shared__ double smem[32 * 8];
  __shared__ T s_alpha[4], s_omega[4];
  __shared__ int s_done[4];
  if (threadIdx.x < 4) {
    s_alpha[threadIdx.x] = (T)F.ks[threadIdx.x].alpha;
    s_omega[threadIdx.x] = (T)F.ks[threadIdx.x].omega;
    s_done[threadIdx.x] = F.ks[threadIdx.x].done;
  }
  __syncthreads();
  if (s_done[0] & s_done[1] & s_done[2] & s_done[3]) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = 1 - pp;
  int c;
  T da[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T db[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  if (interior_index(P, t, c)) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (s_done[s]) continue;
      const T a = s_alpha[s], om = s_omega[s];
      T* x = vec<T>(F.x[s]);
      T* r = vec<T>(F.r[s]);
      const T sv = r[c] - a * vec<T>(F.vk[np][s])[c];
      x[c] = x[c] + a * vec<T>(F.pk[np][s])[c] + om * sv;
      const T rn = sv - om * vec<T>(F.t[s])[c];
      r[c] = rn;
      da[2 * s] = vec<T>(F.rhs[s])[c];
      db[2 * s] = rn;
      da[2 * s + 1] = rn;
      db[2 * s + 1] = rn;
    }
  }
  double part[8];
  block_partial<8>(da, db, part, smem);
  if (publish_is_last<8>(part, F.red, F.counter)) {
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
      F.alg_bytes[HOSC_K_BICG_XR] += launch_bytes(P, s_done, 8.0, 0.0, sizeof(T));
    }
  }
}

// ------------------------------------------------------------------ BiCGSTAB(2), planar FP64
//
// One cycle (Sleijpen and Fokkema's BiCGSTAB(ell) with ell = 2; shadow residual rt = r_0 = rhs)
// in five kernels, each with a last-block reduction that finalises the scalars of the next:
//   B1  u_0 <- r_0 - beta u_0 (on the fly at the stencil), u_1 = A u_0;       alpha = rho/(rt.u_1)
//   B2  r_0 <- r_0 - alpha u_1 (on the fly), r_1 = A r_0; u_0 <- r_0 - beta u_0 and x += alpha u_0
//       (pointwise, with the r_0 of B1);                   rho_1 = rt.r_1, beta = alpha rho_1/rho
//   B3  u_0 <- r_0 - beta u_0 (pointwise); u_1 <- r_1 - beta u_1 (on the fly), u_2 = A u_1;
//                                                          alpha = rho/(rt.u_2)
//   B4  r_0 -= alpha u_1 (pointwise); r_1 <- r_1 - alpha u_2 (on the fly), r_2 = A r_1;
//       x += alpha u_0; the five inner products of r_0, r_1, r_2 give the minimal-residual
//       coefficients: tau = (r_1.r_2)/(r_1.r_1), gamma'_1 = (r_0.r_1)/(r_1.r_1), gamma_2 =
//       gamma'_2 = (r_0.r_2 - tau r_0.r_1)/(r_2.r_2 - tau r_1.r_2), gamma_1 = gamma'_1 - tau gamma_2
//   B5  x += gamma_1 r_0 + gamma_2 r_1; r_0 -= gamma_1 r_1 + gamma_2 r_2; u_0 -= gamma_1 u_1 +
//       gamma_2 u_2 (the Gram-Schmidt step folded into the coefficients); rho <- -omega rho,
//       rho_1 = rt.r_0, beta = alpha rho_1/rho, rho = rho_1, convergence on ||r_0||.
// Buffers per system: r_0 in r / t (ping-pong by cycle: B2 reads one and writes the other, the
// stencil reads the old r_0 at the neighbours), r_1 in pk[0] (B2) then pk[1] (B4), u_1 in vk[0]
// (B1) then vk[1] (B3), u_0, r_2, u_2 in their own arrays. A kernel writes no array that it reads
// at a neighbour.

struct B2Shared {
  double alpha[4], beta[4], g1[4], g2[4];
  int done[4];
};

// The four systems' scalars into shared memory; true when every system is done (uniform).
__device__ __forceinline__ bool b2_load(const Fields& F, B2Shared& sh) {
  if (threadIdx.x < 4) {
    const KrylovScalars k = F.ks[threadIdx.x];
    sh.alpha[threadIdx.x] = k.alpha;
    sh.beta[threadIdx.x] = k.beta;
    sh.g1[threadIdx.x] = k.g1;
    sh.g2[threadIdx.x] = k.g2;
    sh.done[threadIdx.x] = k.done;
  }
  __syncthreads();
  return sh.done[0] & sh.done[1] & sh.done[2] & sh.done[3];
}

__device__ __forceinline__ void nbrs7(int c, int sy, int sz, int nb[7]) {
  nb[0] = c;
  nb[1] = c + 1;
  nb[2] = c - 1;
  nb[3] = c + sy;
  nb[4] = c - sy;
  nb[5] = c + sz;
  nb[6] = c - sz;
}

__device__ __forceinline__ void b2_fail(KrylovScalars& k) {
  k.done = 1;
  k.status = HOSC_ENOCONV;
}

__device__ __forceinline__ const double* const* b2_op(const Fields& F, int s) {
  return (s < 3) ? ops<double>(F.Am) : ops<double>(F.Ae);
}

// B1
__global__ void __launch_bounds__(kThreads) k_b2_u1(DevParams P, Fields F, int cp, int nblocks) {
  __shared__ double smem[32 * 4];
  __shared__ B2Shared sh;
  if (b2_load(F, sh)) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int sy = P.N, sz = P.N * P.N;
  int c;
  double da[4] = {0, 0, 0, 0}, db[4] = {0, 0, 0, 0};
  if (interior_index(P, t, c)) {
    int nb[7];
    nbrs7(c, sy, sz, nb);
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (sh.done[s]) continue;
      const double* r0 = cp ? F.t[s] : F.r[s];
      const double* u0 = F.u0[s];
      const double b = sh.beta[s];
      double un[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) un[q] = r0[nb[q]] - b * u0[nb[q]];
      const double u1 = apply7<double>(b2_op(F, s), c, un[0], un[1], un[2], un[3], un[4], un[5],
                                       un[6]);
      F.vk[0][s][c] = u1;
      da[s] = F.rhs[s][c];
      db[s] = u1;
    }
  }
  double part[4];
  block_partial<4>(da, db, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        if (tot[s] == 0.0 || !isfinite(tot[s])) {
          b2_fail(k);
          continue;
        }
        k.alpha = k.rho / tot[s];
      }
      F.alg_bytes[HOSC_K_BICG_PV] += launch_bytes(P, sh.done, 4.0, 7.0, sizeof(double));
    }
  }
}

// B2
__global__ void __launch_bounds__(kThreads) k_b2_r1(DevParams P, Fields F, int cp, int nblocks) {
  __shared__ double smem[32 * 4];
  __shared__ B2Shared sh;
  if (b2_load(F, sh)) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int sy = P.N, sz = P.N * P.N;
  int c;
  double da[4] = {0, 0, 0, 0}, db[4] = {0, 0, 0, 0};
  if (interior_index(P, t, c)) {
    int nb[7];
    nbrs7(c, sy, sz, nb);
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (sh.done[s]) continue;
      const double* r0 = cp ? F.t[s] : F.r[s];
      double* r0n = cp ? F.r[s] : F.t[s];
      const double* u1 = F.vk[0][s];
      const double a = sh.alpha[s], b = sh.beta[s];
      double rn[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) rn[q] = r0[nb[q]] - a * u1[nb[q]];
      const double r1 = apply7<double>(b2_op(F, s), c, rn[0], rn[1], rn[2], rn[3], rn[4], rn[5],
                                       rn[6]);
      r0n[c] = rn[0];
      F.pk[0][s][c] = r1;
      const double u0 = r0[c] - b * F.u0[s][c];
      F.u0[s][c] = u0;
      F.x[s][c] += a * u0;
      da[s] = F.rhs[s][c];
      db[s] = r1;
    }
  }
  double part[4];
  block_partial<4>(da, db, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        if (k.rho == 0.0 || !isfinite(tot[s])) {
          b2_fail(k);
          continue;
        }
        k.beta = k.alpha * tot[s] / k.rho;
        k.rho = tot[s];
      }
      F.alg_bytes[HOSC_K_BICG_ST] += launch_bytes(P, sh.done, 9.0, 7.0, sizeof(double));
    }
  }
}

// B3
__global__ void __launch_bounds__(kThreads) k_b2_u2(DevParams P, Fields F, int cp, int nblocks) {
  __shared__ double smem[32 * 4];
  __shared__ B2Shared sh;
  if (b2_load(F, sh)) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int sy = P.N, sz = P.N * P.N;
  int c;
  double da[4] = {0, 0, 0, 0}, db[4] = {0, 0, 0, 0};
  if (interior_index(P, t, c)) {
    int nb[7];
    nbrs7(c, sy, sz, nb);
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (sh.done[s]) continue;
      const double* r0 = cp ? F.r[s] : F.t[s];   // written by B2
      const double* r1 = F.pk[0][s];
      const double* u1 = F.vk[0][s];
      const double b = sh.beta[s];
      F.u0[s][c] = r0[c] - b * F.u0[s][c];
      double un[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) un[q] = r1[nb[q]] - b * u1[nb[q]];
      const double u2 = apply7<double>(b2_op(F, s), c, un[0], un[1], un[2], un[3], un[4], un[5],
                                       un[6]);
      F.vk[1][s][c] = un[0];
      F.u2[s][c] = u2;
      da[s] = F.rhs[s][c];
      db[s] = u2;
    }
  }
  double part[4];
  block_partial<4>(da, db, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        if (tot[s] == 0.0 || !isfinite(tot[s])) {
          b2_fail(k);
          continue;
        }
        k.alpha = k.rho / tot[s];
      }
      F.alg_bytes[HOSC_K_BICG_PV] += launch_bytes(P, sh.done, 8.0, 7.0, sizeof(double));
    }
  }
}

// B4
__global__ void __launch_bounds__(kThreads) k_b2_r2(DevParams P, Fields F, int cp, int nblocks) {
  __shared__ double smem[32 * 20];
  __shared__ B2Shared sh;
  if (b2_load(F, sh)) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int sy = P.N, sz = P.N * P.N;
  int c;
  // per system: r1.r1, r1.r2, r2.r2, r0.r1, r0.r2
  double da[20], db[20];
#pragma unroll
  for (int m = 0; m < 20; ++m) da[m] = db[m] = 0.0;
  if (interior_index(P, t, c)) {
    int nb[7];
    nbrs7(c, sy, sz, nb);
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (sh.done[s]) continue;
      double* r0 = cp ? F.r[s] : F.t[s];
      const double* r1 = F.pk[0][s];
      const double* u2 = F.u2[s];
      const double a = sh.alpha[s];
      const double r0c = r0[c] - a * F.vk[1][s][c];
      r0[c] = r0c;
      double rn[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) rn[q] = r1[nb[q]] - a * u2[nb[q]];
      const double r2 = apply7<double>(b2_op(F, s), c, rn[0], rn[1], rn[2], rn[3], rn[4], rn[5],
                                       rn[6]);
      F.pk[1][s][c] = rn[0];
      F.r2[s][c] = r2;
      F.x[s][c] += a * F.u0[s][c];
      const double d0[5] = {rn[0], rn[0], r2, r0c, r0c}, d1[5] = {rn[0], r2, r2, rn[0], r2};
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        da[5 * s + m] = d0[m];
        db[5 * s + m] = d1[m];
      }
    }
  }
  double part[20];
  block_partial<20>(da, db, part, smem);
  if (publish_is_last<20>(part, F.red, F.counter)) {
    double tot[20];
    reduce_partials<20, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        const double* d = tot + 5 * s;   // r1.r1, r1.r2, r2.r2, r0.r1, r0.r2
        const double sig1 = d[0];
        const double tau = sig1 > 0.0 ? d[1] / sig1 : 0.0;
        const double sig2 = d[2] - tau * d[1];   // |r_2 - tau r_1|^2
        if (!(sig1 > 0.0) || !(sig2 > 0.0) || !isfinite(sig2)) {
          b2_fail(k);
          continue;
        }
        const double gp1 = d[3] / sig1, g2 = (d[4] - tau * d[3]) / sig2;
        k.g2 = g2;
        k.g1 = gp1 - tau * g2;
        k.omega = g2;
      }
      F.alg_bytes[HOSC_K_BICG_ST] += launch_bytes(P, sh.done, 10.0, 7.0, sizeof(double));
    }
  }
}

// B5
__global__ void __launch_bounds__(kThreads) k_b2_mr(DevParams P, Fields F, int cp, int nblocks) {
  __shared__ double smem[32 * 8];
  __shared__ B2Shared sh;
  if (b2_load(F, sh)) return;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  int c;
  double da[8] = {0, 0, 0, 0, 0, 0, 0, 0}, db[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (interior_index(P, t, c)) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (sh.done[s]) continue;
      double* r0 = cp ? F.r[s] : F.t[s];
      const double g1 = sh.g1[s], g2 = sh.g2[s];
      const double r0c = r0[c], r1 = F.pk[1][s][c], r2 = F.r2[s][c];
      F.x[s][c] += g1 * r0c + g2 * r1;
      const double rn = r0c - g1 * r1 - g2 * r2;
      r0[c] = rn;
      F.u0[s][c] -= g1 * F.vk[1][s][c] + g2 * F.u2[s][c];
      da[2 * s] = F.rhs[s][c];
      db[2 * s] = rn;
      da[2 * s + 1] = rn;
      db[2 * s + 1] = rn;
    }
  }
  double part[8];
  block_partial<8>(da, db, part, smem);
  if (publish_is_last<8>(part, F.red, F.counter)) {
    double tot[8];
    reduce_partials<8, false>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        const double rho1 = tot[2 * s];
        k.rnorm = sqrt(tot[2 * s + 1]);
        k.iters += 2;
        const double rho0 = -k.omega * k.rho;
        if (k.rnorm <= P.tol_lin * k.r0norm) {
          k.done = 1;
          k.status = 0;
        } else if (!isfinite(k.rnorm) || k.iters >= P.max_lin_iter || rho0 == 0.0) {
          b2_fail(k);
        } else {
          k.beta = k.alpha * rho1 / rho0;
          k.rho = rho1;
        }
      }
      F.alg_bytes[HOSC_K_BICG_XR] += launch_bytes(P, sh.done, 11.0, 0.0, sizeof(double));
    }
  }
}

// ------------------------------------------------------------- merged iteration (two kernels)
//
// The same BiCGSTAB with two kernels per iteration i. k6_a applies the end of iteration i-1
// (s = r - alpha v, x += alpha p + omega s, r_i = s - omega t) and the start of iteration i
// (p_i = r_i + beta (p - omega v), v_i = A p_i) in one pass, recomputing r_i and p_i at the
// stencil's nodes; its partials give rho_i = r_0 . r_i, alpha_i = rho_i / (r_0 . v_i) and the
// true ||r_i|| (the convergence test, one kernel later than in the three-kernel form). k6_b
// computes s, t = A s and the dot products t.s, t.t, r_0.s, r_0.t, from which
// omega_i = t.s / t.t and r_0 . r_{i+1} = r_0.s - omega_i r_0.t follow without another pass;
// then beta_{i+1} = (r_0 . r_{i+1} / rho_i)(alpha_i / omega_i). The residual ping-pongs
// (kr, kr1) since k6_a reads it at the neighbours while writing it.

__global__ void __launch_bounds__(kThreads) k6_init(DevParams P, Fields F) {
  __shared__ double smem[32 * 4];
  const int N = P.N;
  const int n3 = N * N * N;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  FF acc[4] = {};
  if (c < n3) {
    const int i = c % N, j = (c / N) % N, k = c / (N * N);
    const bool inner = i > 0 && j > 0 && k > 0 && i < N - 1 && j < N - 1 && k < N - 1;
    const float4 z = f4(0.f);
    const float4 r = inner ? F.kr0[c] : z;
    F.kr[c] = r;
    F.kr1[c] = z;
    F.kx[c] = z;
    F.kt[c] = z;
    F.kp[0][c] = z;
    F.kp[1][c] = z;
    F.kv[0][c] = z;
    F.kv[1][c] = z;
    ff_dot4(acc, r, r);
  }
  double part[4];
  block_ff<4>(acc, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, gridDim.x, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        k.r0norm = sqrt(tot[s]);
        k.rnorm = k.r0norm;
        k.rho = tot[s];
        k.alpha = 0.0;   // the first k6_a then leaves x = 0, r = r_0 and sets p = r_0
        k.omega = 0.0;
        k.beta = 0.0;
        k.iters = 0;
        k.pad = 0;       // no x, r update applied yet
        k.status = 0;
        // an inner pressure pass solves the momentum systems only
        k.done = (k.r0norm == 0.0 || *F.halt || (s == 3 && P.inner_pass)) ? 1 : 0;
      }
    }
  }
}

template <int MinB>
__global__ void __launch_bounds__(256, MinB) k6_a(DevParams P, Fields F, int pp) {
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return;   // uniform over the grid
  const bool ene = !sc.done[3];   // the energy system still iterates (uniform)
  const int N = P.N, N2 = N * N;
  const float4 a = sc.a, ma = neg4(sc.a), om = sc.om, mom = neg4(sc.om), b = sc.b;
  const float4* __restrict__ Ro = pp ? F.kr1 : F.kr;
  float4* __restrict__ Rn = pp ? F.kr : F.kr1;
  const float4* __restrict__ Vo = F.kv[pp];
  const float4* __restrict__ Po = F.kp[pp];
  const float4* __restrict__ T = F.kt;
  auto pnew = [&](int c) {
    const float4 v = __ldg(Vo + c);
    const float4 rn = fma4(mom, __ldg(T + c), fma4(ma, v, __ldg(Ro + c)));
    return fma4(b, fma4(mom, v, __ldg(Po + c)), rn);
  };
  FF acc[12] = {};
  Column col;
  if (column(P, col)) {
    float4 pm = pnew(col.cb + N2 * (col.k0 - 1));
    float4 pc = pnew(col.cb + N2 * col.k0);
    for (int k = col.k0; k < col.k1; ++k) {
      const int c = col.cb + N2 * k;
      const float4 pz = pnew(c + N2);
      const float4 vn = apply_op(P, load_op(F, c, ene), pc, pnew(c + 1), pnew(c - 1),
                                 pnew(c + N), pnew(c - N), pz, pm);
      const float4 r = __ldg(Ro + c), v = __ldg(Vo + c), p = __ldg(Po + c);
      const float4 sv = fma4(ma, v, r);
      const float4 rn = fma4(mom, __ldg(T + c), sv);
      F.kx[c] = fma4(om, sv, fma4(a, p, F.kx[c]));
      Rn[c] = rn;
      F.kp[1 - pp][c] = pc;
      F.kv[1 - pp][c] = vn;
      const float4 r0 = __ldg(F.kr0 + c);
      ff_dot4(acc, r0, vn);
      ff_dot4(acc + 4, rn, rn);
      ff_dot4(acc + 8, r0, rn);
      pm = pc;
      pc = pz;
    }
  }
  double part[12];
  block_ff<12>(acc, part, smem);
  if (publish_is_last<12>(part, F.red, F.counter, block_id(), block_count())) {
    double tot[12];
    reduce_partials<12, false>(tot, F.red, block_count(), F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        k.rnorm = sqrt(tot[4 + s]);
        if (k.pad) k.iters += 1;
        k.pad = 1;
        if (k.rnorm <= P.tol_lin * k.r0norm) {
          k.done = 1;
          k.status = 0;
          continue;
        }
        if (!isfinite(k.rnorm) || k.iters >= P.max_lin_iter || tot[s] == 0.0 ||
            !isfinite(tot[s])) {
          k.done = 1;
          k.status = HOSC_ENOCONV;
          continue;
        }
        k.rho = tot[8 + s];   // rho_i = r_0 . r_i from the stored r_i
        k.alpha = k.rho / tot[s];
      }
      // r p v t x r0 in, x r p v out, the compact operators
      F.alg_bytes[HOSC_K_BICG_PV] += bytes4(P, 10.0 + op_words(ene));
    }
  }
}

template <int MinB>
__global__ void __launch_bounds__(256, MinB) k6_b(DevParams P, Fields F, int pp) {
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return;
  const bool ene = !sc.done[3];   // the energy system still iterates (uniform)
  const int N = P.N, N2 = N * N;
  const float4 ma = neg4(sc.a);
  const float4* __restrict__ R = pp ? F.kr : F.kr1;   // r_i, written by k6_a
  const float4* __restrict__ V = F.kv[1 - pp];
  auto sval = [&](int c) { return fma4(ma, __ldg(V + c), __ldg(R + c)); };
  FF acc[16] = {};
  Column col;
  if (column(P, col)) {
    float4 sm = sval(col.cb + N2 * (col.k0 - 1));
    float4 sc0 = sval(col.cb + N2 * col.k0);
    for (int k = col.k0; k < col.k1; ++k) {
      const int c = col.cb + N2 * k;
      const float4 sz = sval(c + N2);
      const float4 tv = apply_op(P, load_op(F, c, ene), sc0, sval(c + 1), sval(c - 1),
                                 sval(c + N), sval(c - N), sz, sm);
      F.kt[c] = tv;
      const float4 r0 = __ldg(F.kr0 + c);
      ff_dot4(acc, tv, sc0);
      ff_dot4(acc + 4, tv, tv);
      ff_dot4(acc + 8, r0, sc0);
      ff_dot4(acc + 12, r0, tv);
      sm = sc0;
      sc0 = sz;
    }
  }
  double part[16];
  block_ff<16>(acc, part, smem);
  if (publish_is_last<16>(part, F.red, F.counter, block_id(), block_count())) {
    double tot[16];
    reduce_partials<16, false>(tot, F.red, block_count(), F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        const double ts = tot[s], tt = tot[4 + s], r0s = tot[8 + s], r0t = tot[12 + s];
        const double om = tt > 0.0 ? ts / tt : 0.0;
        const double rho_next = r0s - om * r0t;   // r_0 . (s - omega t) = r_0 . r_{i+1}
        if (om == 0.0 || rho_next == 0.0 || !isfinite(rho_next)) {
          k.done = 1;
          k.status = HOSC_ENOCONV;
          continue;
        }
        // k6_a recomputes rho_{i+1} from the stored r_{i+1}; this value only sets beta
        k.beta = (rho_next / k.rho) * (k.alpha / om);
        k.omega = om;
      }
      // r v r0 in, t out, the compact operators
      F.alg_bytes[HOSC_K_BICG_ST] += bytes4(P, 4.0 + op_words(ene));
    }
  }
}

// ------------------------------------------------------- staged stencil kernels (cp.async)
//
// The p/v and s/t kernels again, with their reads staged through shared memory. A block owns a
// tile of sx * sy interior columns (one thread each) and a segment of skz planes. The planes it
// needs (the haloed tile of each stencil vector, and the weights and r_0 at the tile's nodes)
// stream through a ring of kStages shared-memory stages with cp.async: 16-byte copies from global
// to shared memory that hold no registers while in flight. While plane k is computed (from the
// stages of planes k and k+1; plane k-1 is held in registers), planes k+2 and k+3 are in flight.
// The stencil reads shared memory only.

constexpr int kStages = 4;

__device__ __forceinline__ void cp_async16(float4* smem_dst, const float4* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 16 : 0;   // 0: write zeros, read nothing
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_two() {   // all but the two newest groups have landed
  asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc), "r"(n)
               : "memory");
}

// Shared-memory layout of one stage, in float4: NV haloed vectors ((sx+2)(sy+2) each), then the
// compact operators of the tile's nodes (momentum float4s, energy float4s, then L as floats in
// ceil(sx*sy/4) float4 slots), then (p/v only) r_0 of the tile.
struct StageLayout {
  int hx, halo, tile, nv, lslots, per_stage;
  __host__ __device__ StageLayout(int sx, int sy, int nvec, bool with_r0) {
    hx = sx + 2;
    halo = (sx + 2) * (sy + 2);
    tile = sx * sy;
    nv = nvec;
    lslots = (tile + 3) / 4;
    per_stage = nv * halo + 2 * tile + lslots + (with_r0 ? tile : 0);
  }
  __host__ __device__ int op_m() const { return nv * halo; }
  __host__ __device__ int op_e() const { return nv * halo + tile; }
  __host__ __device__ int op_l() const { return nv * halo + 2 * tile; }
  __host__ __device__ int r0() const { return nv * halo + 2 * tile + lslots; }
};

// Copy plane q (if it exists for this block) into stage buffer st: the haloed tile of each
// stencil vector, then the compact operators (and r_0) at the tile's interior nodes; the energy
// operator only while that system iterates. Positions outside the grid are zero-filled without
// a read; the data of this plane form one commit group.
template <int NV, bool R0>
__device__ __forceinline__ void stage_plane(float4* st, const StageLayout& L, int N, int i0,
                                            int j0, int q, bool live,
                                            const float4* const (&vecs)[NV], const Fields& F,
                                            bool ene, int sx) {
  if (live) {
    const int nthr = blockDim.x;
    for (int idx = threadIdx.x; idx < L.halo; idx += nthr) {
      const int hy = idx / L.hx, hx = idx - hy * L.hx;
      const int gi = i0 - 1 + hx, gj = j0 - 1 + hy;
      const bool ok = gi <= N - 1 && gj <= N - 1;
      const int off = ok ? gi + N * (gj + N * q) : 0;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async16(st + v * L.halo + idx, vecs[v] + off, ok);
    }
    const bool inner_plane = q >= 1 && q <= N - 2;
    for (int e = threadIdx.x; e < L.tile; e += nthr) {
      const int ty = e / sx, tx = e - ty * sx;
      const int gi = i0 + tx, gj = j0 + ty;
      const bool ok = inner_plane && gi <= N - 2 && gj <= N - 2;
      const int off = ok ? gi + N * (gj + N * q) : 0;
      cp_async16(st + L.op_m() + e, F.kwm + off, ok);
      cp_async16(st + L.op_e() + e, F.kwe + off, ok && ene);
      cp_async4((float*)(st + L.op_l()) + e, F.kL + off, ok);
      if (R0) cp_async16(st + L.r0() + e, F.kr0 + off, ok);
    }
  }
  cp_commit();   // one group per plane, empty past the segment
}

__device__ __forceinline__ Op4 staged_op(const float4* sq, const StageLayout& L, int t) {
  Op4 op;
  op.m = sq[L.op_m() + t];
  op.e = sq[L.op_e() + t];
  op.l12 = ((const float*)(sq + L.op_l()))[t] * (1.f / 12.f);
  return op;
}

// Staged p/v kernel (same arithmetic as k4_pv).
__global__ void __launch_bounds__(256) k5_pv(DevParams P, Fields F, int pp) {
  extern __shared__ float4 ring[];
  __shared__ double smem[32 * 4];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return;
  const int N = P.N, N2 = N * N, sx = P.sx;
  const StageLayout L(sx, P.sy, 3, true);
  const int i0 = 1 + blockIdx.x * sx, j0 = 1 + blockIdx.y * P.sy;
  const int k0 = 1 + blockIdx.z * P.skz, k1 = min(k0 + P.skz, N - 1);
  const int t = threadIdx.x, ty = t / sx, tx = t - ty * sx;
  const bool mine = ty < P.sy && i0 + tx <= N - 2 && j0 + ty <= N - 2;
  const int h = (ty + 1) * L.hx + (tx + 1);
  const float4 b = sc.b, mom = neg4(sc.om);
  const float4* const vecs[3] = {F.kr, F.kp[pp], F.kv[pp]};
  const bool ene = !sc.done[3];
  auto stage_of = [&](int q) { return ring + ((q - (k0 - 1)) % kStages) * L.per_stage; };
  auto pnew = [&](const float4* st, int idx) {
    return fma4(b, fma4(mom, st[2 * L.halo + idx], st[L.halo + idx]), st[idx]);
  };
  // planes k0-1 .. k0+2 in flight; wait for the first two
  for (int q = k0 - 1; q <= k0 + 2; ++q)
    stage_plane<3, true>(stage_of(q), L, N, i0, j0, q, q <= k1, vecs, F, ene, sx);
  cp_wait_two();
  __syncthreads();
  float4 pm = pnew(stage_of(k0 - 1), h), pc = pnew(stage_of(k0), h);
  __syncthreads();   // the stage of plane k0-1 is free for plane k0+3
  FF acc[4] = {};
  for (int k = k0; k < k1; ++k) {
    stage_plane<3, true>(stage_of(k + 3), L, N, i0, j0, k + 3, k + 3 <= k1, vecs, F, ene, sx);
    cp_wait_two();   // plane k+1 has landed
    __syncthreads();
    const float4* sq = stage_of(k);
    const float4 pz = pnew(stage_of(k + 1), h);
    if (mine) {
      const float4 vn = apply_op(P, staged_op(sq, L, t), pc, pnew(sq, h + 1), pnew(sq, h - 1),
                                 pnew(sq, h + L.hx), pnew(sq, h - L.hx), pz, pm);
      const int c = (i0 + tx) + N * (j0 + ty) + N2 * k;
      F.kp[1 - pp][c] = pc;
      F.kv[1 - pp][c] = vn;
      ff_dot4(acc, sq[L.r0() + t], vn);
    }
    pm = pc;
    pc = pz;
    __syncthreads();   // the stage of plane k is free for plane k+4
  }
  double part[4];
  block_ff<4>(acc, part, smem);
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  if (publish_is_last<4>(part, F.red, F.counter, bid, nb)) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, nb, F.counter, smem);
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
      F.alg_bytes[HOSC_K_BICG_PV] += bytes4(P, 6.0 + op_words(ene));
    }
  }
}

// Staged s/t kernel (same arithmetic as k4_st).
__global__ void __launch_bounds__(256) k5_st(DevParams P, Fields F, int pp) {
  extern __shared__ float4 ring[];
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return;
  const int N = P.N, N2 = N * N, sx = P.sx;
  const StageLayout L(sx, P.sy, 2, false);
  const int i0 = 1 + blockIdx.x * sx, j0 = 1 + blockIdx.y * P.sy;
  const int k0 = 1 + blockIdx.z * P.skz, k1 = min(k0 + P.skz, N - 1);
  const int t = threadIdx.x, ty = t / sx, tx = t - ty * sx;
  const bool mine = ty < P.sy && i0 + tx <= N - 2 && j0 + ty <= N - 2;
  const int h = (ty + 1) * L.hx + (tx + 1);
  const float4 ma = neg4(sc.a);
  const float4* const vecs[2] = {F.kr, F.kv[1 - pp]};
  const bool ene = !sc.done[3];
  auto stage_of = [&](int q) { return ring + ((q - (k0 - 1)) % kStages) * L.per_stage; };
  auto sval = [&](const float4* st, int idx) { return fma4(ma, st[L.halo + idx], st[idx]); };
  for (int q = k0 - 1; q <= k0 + 2; ++q)
    stage_plane<2, false>(stage_of(q), L, N, i0, j0, q, q <= k1, vecs, F, ene, sx);
  cp_wait_two();
  __syncthreads();
  float4 sm = sval(stage_of(k0 - 1), h), sc0 = sval(stage_of(k0), h);
  __syncthreads();
  FF acc[8] = {};
  for (int k = k0; k < k1; ++k) {
    stage_plane<2, false>(stage_of(k + 3), L, N, i0, j0, k + 3, k + 3 <= k1, vecs, F, ene, sx);
    cp_wait_two();
    __syncthreads();
    const float4* sq = stage_of(k);
    const float4 sz = sval(stage_of(k + 1), h);
    if (mine) {
      const float4 tv = apply_op(P, staged_op(sq, L, t), sc0, sval(sq, h + 1), sval(sq, h - 1),
                                 sval(sq, h + L.hx), sval(sq, h - L.hx), sz, sm);
      const int c = (i0 + tx) + N * (j0 + ty) + N2 * k;
      F.kt[c] = tv;
      ff_dot4(acc, tv, sc0);
      ff_dot4(acc + 4, tv, tv);
    }
    sm = sc0;
    sc0 = sz;
    __syncthreads();
  }
  double part[8];
  block_ff<8>(acc, part, smem);
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  if (publish_is_last<8>(part, F.red, F.counter, bid, nb)) {
    double tot[8];
    reduce_partials<8, false>(tot, F.red, nb, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        k.omega = tot[4 + s] > 0.0 ? tot[s] / tot[4 + s] : 0.0;
      }
      F.alg_bytes[HOSC_K_BICG_ST] += bytes4(P, 3.0 + op_words(ene));
    }
  }
}

dim3 grid5(const DevParams& P) {
  const int ni = P.N - 2;
  return dim3((unsigned)((ni + P.sx - 1) / P.sx), (unsigned)((ni + P.sy - 1) / P.sy),
              (unsigned)((ni + P.skz - 1) / P.skz));
}

dim3 grid4(const DevParams& P) {
  const int ni = P.N - 2;
  return dim3((unsigned)((ni * ni + P.kblock - 1) / P.kblock), (unsigned)((ni + P.kz - 1) / P.kz));
}

int interior_blocks(const DevParams& P) {
  const long ni = P.N - 2;
  return red_blocks(ni * ni * ni);
}

}  // namespace

namespace {
__global__ void k_krylov_activate(KrylovScalars* ks) {
  if (threadIdx.x < 4) {
    ks[threadIdx.x].done = 0;
    ks[threadIdx.x].iters = 0;
    ks[threadIdx.x].status = 0;
  }
}
}  // namespace

void launch_krylov_activate(const Fields& F, cudaStream_t s) {
  k_krylov_activate<<<1, 32, 0, s>>>(F.ks);
}

void launch_loop_cond(const Fields& F, unsigned long long handle, cudaStream_t s) {
  k_loop_cond<<<1, 32, 0, s>>>(F.ks, (cudaGraphConditionalHandle)handle);
}

void launch_bicg_init(const DevParams& P, const Fields& F, cudaStream_t s) {
  if (P.krylov_fp32 && P.merged) {
    const long n3 = (long)P.N * P.N * P.N;
    k6_init<<<red_blocks(n3), kThreads, 0, s>>>(P, F);
    return;
  }
  if (P.krylov_fp32) {
    const long n3 = (long)P.N * P.N * P.N;
    const int most = 8 * device_sms();   // resident blocks of one wave
    const int b = red_blocks(n3) < most ? red_blocks(n3) : most;
    k4_init<<<b, kThreads, 0, s>>>(P, F);
    return;
  }
  const int b = interior_blocks(P);
  k_bicg_init<double><<<b, kThreads, 0, s>>>(P, F, b);
}

// x/r as one flat stream: every node of the interior planes, the i and j walls included (every
// vector is zero there: the workspace is zeroed at creation, k4_init zeroes x, r, p and v
// everywhere, and no kernel writes the wall entries of t or r_0), in a grid-stride loop that
// issues the loads of U nodes before their arithmetic, so that a thread keeps 6 U float4 loads in
// flight. Same arithmetic and float-float partials as k4_xr; one block partial per block.
template <int U>
__global__ void __launch_bounds__(256) k8_xr(DevParams P, Fields F, int pp) {
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  pdl_wait_and_release();
  load_scalars(F.ks, sc);
  if (sc.all_done) return;
  const int np = 1 - pp;
  const float4 a = sc.a, om = sc.om, ma = neg4(sc.a), mom = neg4(sc.om);
  const float4* __restrict__ V = F.kv[np];
  const float4* __restrict__ Pv = F.kp[np];
  const float4* __restrict__ T = F.kt;
  const float4* __restrict__ R0 = F.kr0;
  float4* __restrict__ X = F.kx;
  float4* __restrict__ R = F.kr;
  const unsigned N2 = (unsigned)P.N * (unsigned)P.N, hi = N2 * (unsigned)(P.N - 1);
  const unsigned stride = gridDim.x * blockDim.x;
  FF acc[8] = {};
  unsigned c = N2 + blockIdx.x * blockDim.x + threadIdx.x;
  for (; c + (U - 1) * stride < hi; c += U * stride) {
    float4 r[U], v[U], p[U], t[U], r0[U], x[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const unsigned e = c + q * stride;
      r[q] = R[e];
      x[q] = X[e];
      v[q] = __ldg(V + e);
      p[q] = __ldg(Pv + e);
      t[q] = __ldg(T + e);
      r0[q] = __ldg(R0 + e);
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const unsigned e = c + q * stride;
      const float4 sv = fma4(ma, v[q], r[q]);
      X[e] = fma4(om, sv, fma4(a, p[q], x[q]));
      const float4 rn = fma4(mom, t[q], sv);
      R[e] = rn;
      ff_dot4(acc, r0[q], rn);
      ff_dot4(acc + 4, rn, rn);
    }
  }
  for (; c < hi; c += stride) {
    const float4 sv = fma4(ma, __ldg(V + c), R[c]);
    X[c] = fma4(om, sv, fma4(a, __ldg(Pv + c), X[c]));
    const float4 rn = fma4(mom, __ldg(T + c), sv);
    R[c] = rn;
    ff_dot4(acc, __ldg(R0 + c), rn);
    ff_dot4(acc + 4, rn, rn);
  }
  double part[8];
  block_ff<8>(acc, part, smem);
  if (publish_is_last<8>(part, F.red, F.counter, blockIdx.x, gridDim.x))
    xr_finish(P, F, gridDim.x, smem);
}

// Blocks of the flat x/r kernel: resident blocks of one wave.
int xr_flat_blocks() {
  static int occ = 0;
  if (occ == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k8_xr<4>, 256, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 4;
    }
  }
  return occ * device_sms();
}


// Launch of an interleaved Krylov kernel with programmatic stream serialisation (see
// pdl_wait_and_release): in a captured step the kernels of the BiCGSTAB loop chain with
// programmatic edges.
template <class K>
void launch_pdl(K kern, dim3 grid, int threads, cudaStream_t s, const DevParams& P,
                const Fields& F, int pp) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, P, F, pp);
}

void launch_bicg_pv(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  if (P.krylov_fp32 && P.merged) {   // x, r update of the previous iteration, then p, v
    if (P.narrow) k6_a<4><<<grid4(P), P.kblock, 0, s>>>(P, F, pp);
    else k6_a<2><<<grid4(P), P.kblock, 0, s>>>(P, F, pp);
    return;
  }
  if (P.krylov_fp32 && P.tty > 0 && (P.tkernels & 1)) {
    launch_tma_pv(P, F, pp, s);
    return;
  }
  if (P.krylov_fp32 && P.sx > 0) {
    k5_pv<<<grid5(P), P.sx * P.sy, staged_smem_bytes(P.sx, P.sy, true), s>>>(P, F, pp);
    return;
  }
  if (P.krylov_fp32) {
    if (P.narrow) launch_pdl(k4_pv<4>, grid4(P), P.kblock, s, P, F, pp);
    else launch_pdl(k4_pv<2>, grid4(P), P.kblock, s, P, F, pp);
    return;
  }
  const int b = interior_blocks(P);
  k_bicg_pv<double><<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_bicg_st(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  if (P.krylov_fp32 && P.merged) {
    if (P.narrow) k6_b<4><<<grid4(P), P.kblock, 0, s>>>(P, F, pp);
    else k6_b<2><<<grid4(P), P.kblock, 0, s>>>(P, F, pp);
    return;
  }
  if (P.krylov_fp32 && P.tty > 0 && (P.tkernels & 2)) {
    launch_tma_st(P, F, pp, s);
    return;
  }
  if (P.krylov_fp32 && P.sx > 0) {
    k5_st<<<grid5(P), P.sx * P.sy, staged_smem_bytes(P.sx, P.sy, false), s>>>(P, F, pp);
    return;
  }
  if (P.krylov_fp32) {
    if (P.narrow) launch_pdl(k4_st<4>, grid4(P), P.kblock, s, P, F, pp);
    else launch_pdl(k4_st<2>, grid4(P), P.kblock, s, P, F, pp);
    return;
  }
  const int b = interior_blocks(P);
  k_bicg_st<double><<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_bicg_xr(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  if (P.krylov_fp32 && P.merged) return;   // folded into the next k6_a
  if (P.krylov_fp32 && P.xr_flat) {
    launch_pdl(k8_xr<4>, dim3(xr_flat_blocks()), 256, s, P, F, pp);
    return;
  }
  if (P.krylov_fp32) {
    if (P.narrow) launch_pdl(k4_xr<4>, grid4(P), P.kblock, s, P, F, pp);
    else launch_pdl(k4_xr<2>, grid4(P), P.kblock, s, P, F, pp);
    return;
  }
  const int b = interior_blocks(P);
  k_bicg_xr<double><<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_b2(int kernel, const DevParams& P, const Fields& F, int cp, cudaStream_t s) {
  const int b = interior_blocks(P);
  switch (kernel) {
    case 0: k_b2_u1<<<b, kThreads, 0, s>>>(P, F, cp, b); break;
    case 1: k_b2_r1<<<b, kThreads, 0, s>>>(P, F, cp, b); break;
    case 2: k_b2_u2<<<b, kThreads, 0, s>>>(P, F, cp, b); break;
    case 3: k_b2_r2<<<b, kThreads, 0, s>>>(P, F, cp, b); break;
    default: k_b2_mr<<<b, kThreads, 0, s>>>(P, F, cp, b); break;
  }
}

long krylov4_blocks(const DevParams& P) {
  const dim3 g = grid4(P);
  long nb = (long)g.x * g.y;
  if (P.sx > 0) {
    const dim3 g5 = grid5(P);
    const long n5 = (long)g5.x * g5.y * g5.z;
    nb = n5 > nb ? n5 : nb;
  }
  const long n7 = tma_blocks(P);
  return n7 > nb ? n7 : nb;
}

size_t staged_smem_bytes(int sx, int sy, bool pv) {
  const StageLayout L(sx, sy, pv ? 3 : 2, pv);
  return (size_t)kStages * L.per_stage * sizeof(float4);
}

// Opt the staged kernels in to large dynamic shared memory (once per device and process).
bool staged_smem_ready() {
  static int done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (!done[dev]) {
    const int cap = 200 * 1024;
    if (cudaFuncSetAttribute(k5_pv, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k5_st, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    done[dev] = 1;
  }
  return true;
}

double staged_wave_cost(int N, int sx, int sy, int skz, int sms) {
  if (!staged_smem_ready()) return 1e300;
  const size_t smem = staged_smem_bytes(sx, sy, true);
  if (smem > 200 * 1024) return 1e300;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k5_pv, sx * sy, smem) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return 1e300;
  }
  const long ni = N - 2;
  const long items = ((ni + sx - 1) / sx) * ((ni + sy - 1) / sy) * ((ni + skz - 1) / skz);
  const long slots = (long)occ * sms;
  const long waves = (items + slots - 1) / slots;
  return (double)waves * (skz + 2);
}

int krylov4_occupancy(int kblock, int narrow, int merged) {
  int occ = 0;
  cudaError_t e;
  if (merged)
    e = narrow ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k6_a<4>, kblock, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k6_a<2>, kblock, 0);
  else
    e = narrow ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k4_pv<4>, kblock, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k4_pv<2>, kblock, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return occ > 0 ? occ : 1;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return sms > 0 ? sms : 152;
}

double krylov4_wave_cost(int N, int kblock, int kz, int narrow, int merged, int sms) {
  const long ni = N - 2;
  const long items = ((ni * ni + kblock - 1) / kblock) * ((ni + kz - 1) / kz);
  const long slots = (long)krylov4_occupancy(kblock, narrow, merged) * sms;
  const long waves = (items + slots - 1) / slots;
  // every resident block streams kz planes plus the two it reads around its segment
  return (double)waves * (kz + 2);
}

void default_tiles(int N, int* kblock, int* kz) {
  const int sms = device_sms();
  const int ni = N - 2;
  double best = 1e300;
  int bb = 128, bz = 1;
  for (int z = 1; z <= (ni < 16 ? ni : 16); ++z) {
    const double c = krylov4_wave_cost(N, 128, z, 0, 0, sms);
    if (c < best) {
      best = c;
      bz = z;
    }
  }
  *kblock = bb;
  *kz = bz;
}

}  // namespace hosc
