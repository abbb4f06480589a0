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

// Float-float ("double-float") numbers: an unevaluated sum hi + lo of two floats. Knuth's TwoSum
// and an FMA-based exact product give sums with about 44 significant bits using float
// instructions only, which GB300 issues at 64x the rate of double instructions.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_prod(float a, float b) {
  FF r;
  r.hi = a * b;
  r.lo = fmaf(a, b, -r.hi);   // exact rounding error of the product
  return r;
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);   // TwoSum: s + err == a.hi + b.hi exactly
  const float lo = err + a.lo + b.lo;
  FF r;
  r.hi = s + lo;
  r.lo = lo - (r.hi - s);
  return r;
}

__device__ __forceinline__ FF ff_shfl_down(FF a, int off) {
  FF r;
  r.hi = __shfl_down_sync(0xffffffffu, a.hi, off);
  r.lo = __shfl_down_sync(0xffffffffu, a.lo, off);
  return r;
}

// Block partial of M dot-product terms a[m] * b[m]. For float vectors the products and the warp
// and cross-warp sums are float-float (no double instruction per thread) and thread 0 widens the
// block total to double; for double vectors every stage is double. The grid stage in the last
// block adds the block totals in double. The result is valid in thread 0.
template <class T, int M>
__device__ __forceinline__ void block_partial(const T (&a)[M], const T (&b)[M], double (&out)[M],
                                              double* smem) {
  if constexpr (sizeof(T) == sizeof(float)) {
    FF* fs = reinterpret_cast<FF*>(smem);
    FF w[M];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      w[m] = ff_prod(a[m], b[m]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) w[m] = ff_add(w[m], ff_shfl_down(w[m], off));
    }
    if (lane == 0) {
#pragma unroll
      for (int m = 0; m < M; ++m) fs[wid * M + m] = w[m];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        FF x = (lane < nw) ? fs[lane * M + m] : FF{0.0f, 0.0f};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = ff_add(x, ff_shfl_down(x, off));
        if (lane == 0) out[m] = (double)x.hi + (double)x.lo;
      }
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) out[m] = (double)a[m] * (double)b[m];
    block_reduce<M, false>(out, smem);
  }
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
      da[s] = r;
      db[s] = r;
    }
  }
  double part[4];
  block_partial<T, 4>(da, db, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter)) {
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
        k.done = (k.r0norm == 0.0 || *F.halt) ? 1 : 0;
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
  block_partial<T, 4>(da, db, part, smem);
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
  block_partial<T, 8>(da, db, part, smem);
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
  block_partial<T, 8>(da, db, part, smem);
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

int interior_blocks(const DevParams& P) {
  const long ni = P.N - 2;
  return red_blocks(ni * ni * ni);
}

}  // namespace

void launch_loop_cond(const Fields& F, unsigned long long handle, cudaStream_t s) {
  k_loop_cond<<<1, 32, 0, s>>>(F.ks, (cudaGraphConditionalHandle)handle);
}

void launch_bicg_init(const DevParams& P, const Fields& F, cudaStream_t s) {
  const int b = interior_blocks(P);
  if (P.krylov_fp32) k_bicg_init<float><<<b, kThreads, 0, s>>>(P, F, b);
  else k_bicg_init<double><<<b, kThreads, 0, s>>>(P, F, b);
}

void launch_bicg_pv(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  const int b = interior_blocks(P);
  if (P.krylov_fp32) k_bicg_pv<float><<<b, kThreads, 0, s>>>(P, F, pp, b);
  else k_bicg_pv<double><<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_bicg_st(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  const int b = interior_blocks(P);
  if (P.krylov_fp32) k_bicg_st<float><<<b, kThreads, 0, s>>>(P, F, pp, b);
  else k_bicg_st<double><<<b, kThreads, 0, s>>>(P, F, pp, b);
}

void launch_bicg_xr(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  const int b = interior_blocks(P);
  if (P.krylov_fp32) k_bicg_xr<float><<<b, kThreads, 0, s>>>(P, F, pp, b);
  else k_bicg_xr<double><<<b, kThreads, 0, s>>>(P, F, pp, b);
}

}  // namespace hosc
