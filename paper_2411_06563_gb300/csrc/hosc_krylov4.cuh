// Device code of the interleaved FP32 BiCGSTAB of the mixed-precision solve (Punia & Ray,
// arXiv:2411.06563, Sec. 2.2: unpreconditioned BiCGSTAB on the four level-(n+1) systems): one
// float4 per node holds the u, v, w, theta values of a vector, the operators are the compact
// float forms written by the right-hand-side kernel, and a thread owns one interior (i, j) column
// over a segment of kz planes, keeping the z-neighbours in registers as it marches; dot-product
// terms accumulate in float-float over the segment before the block reduction, and the last
// block of a launch (a ticket counter) finalises the scalars the next kernel needs.
//
// The kernels are device bodies taking the block's (virtual) position in the grid of column chunks
// and plane segments, so that the per-kernel launches (hosc_krylov.cu) and the persistent round
// kernel of the pool (hosc_round.cu) run the same code.
#pragma once

#include <math.h>

#include "hosc_device.cuh"
#include "hosc_internal.h"

namespace hosc {

namespace {

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

// Block sum of M per-thread float-float accumulators; thread 0 receives the totals in double.
template <int M>
__device__ __forceinline__ void block_ff(FF (&acc)[M], double (&out)[M], double* smem) {
  FF* fs = reinterpret_cast<FF*>(smem);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int m = 0; m < M; ++m) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[m] = ff_add(acc[m], ff_shfl_down(acc[m], off));
  }
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) fs[wid * M + m] = acc[m];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      FF x = (lane < nw) ? fs[lane * M + m] : FF{0.0f, 0.0f};
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x = ff_add(x, ff_shfl_down(x, off));
      out[m] = (double)x.hi + (double)x.lo;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ interleaved FP32 solve

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }

// a + b * c per component
__device__ __forceinline__ float4 fma4(float4 b, float4 c, float4 a) {
  return make_float4(fmaf(b.x, c.x, a.x), fmaf(b.y, c.y, a.y), fmaf(b.z, c.z, a.z),
                     fmaf(b.w, c.w, a.w));
}
__device__ __forceinline__ float4 neg4(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

// acc[m0 + s] += a_s * b_s for the four systems s
__device__ __forceinline__ void ff_dot4(FF* acc, float4 a, float4 b) {
  acc[0] = ff_add(acc[0], ff_prod(a.x, b.x));
  acc[1] = ff_add(acc[1], ff_prod(a.y, b.y));
  acc[2] = ff_add(acc[2], ff_prod(a.z, b.z));
  acc[3] = ff_add(acc[3], ff_prod(a.w, b.w));
}

// The seven-point operators of the four systems at node c, from the compact operators: along
// direction d the +d and -d neighbours weigh S_d - B_d and S_d + B_d, so the product is
// D o + sum_d S_d (o_{+d} + o_{-d}) - B_d (o_{+d} - o_{-d}). Momentum (u, v, w lanes): B and D from
// kwm, S_d = -dt/(2 h_d^2) + L/12. Energy (theta lane): B and D from kwe, S_d = -dt/(2 h_d^2) +
// 1/12; with ene false (the energy system has converged) its weights are not read and the lane
// is zero. With Jacobi row scaling (precond) each row is divided by its diagonal D.
struct Op4 {
  float4 m, e;   // (B_x, B_y, B_z, D) of momentum and of energy
  float l12;     // L/12
};

__device__ __forceinline__ Op4 load_op(const Fields& F, int c, bool ene) {
  Op4 op;
  op.m = HOSC_LDG(F.kwm + c);
  op.l12 = HOSC_LDG(F.kL + c) * (1.f / 12.f);
  op.e = ene ? HOSC_LDG(F.kwe + c) : make_float4(0.f, 0.f, 0.f, 0.f);
  return op;
}

__device__ __forceinline__ float4 apply_op(const DevParams& P, const Op4& op, float4 o, float4 xp,
                                           float4 xm, float4 yp, float4 ym, float4 zp,
                                           float4 zm) {
  // momentum weights of the six neighbours, shared by the u, v, w lanes
  const float Sx = P.csf[0] + op.l12, Sy = P.csf[1] + op.l12, Sz = P.csf[2] + op.l12;
  const float4 m = op.m, e = op.e;
  const float a1 = Sx - m.x, a2 = Sx + m.x, a3 = Sy - m.y, a4 = Sy + m.y, a5 = Sz - m.z,
              a6 = Sz + m.z;
  float4 y;
  y.x = m.w * o.x + a1 * xp.x + a2 * xm.x + a3 * yp.x + a4 * ym.x + a5 * zp.x + a6 * zm.x;
  y.y = m.w * o.y + a1 * xp.y + a2 * xm.y + a3 * yp.y + a4 * ym.y + a5 * zp.y + a6 * zm.y;
  y.z = m.w * o.z + a1 * xp.z + a2 * xm.z + a3 * yp.z + a4 * ym.z + a5 * zp.z + a6 * zm.z;
  const float c12 = 1.f / 12.f;
  const float ex = P.csf[0] + c12, ey = P.csf[1] + c12, ez = P.csf[2] + c12;
  y.w = e.w * o.w + (ex - e.x) * xp.w + (ex + e.x) * xm.w + (ey - e.y) * yp.w +
        (ey + e.y) * ym.w + (ez - e.z) * zp.w + (ez + e.z) * zm.w;
  if (P.precond) {
    const float im = 1.f / m.w;
    y.x *= im;
    y.y *= im;
    y.z *= im;
    y.w = e.w != 0.f ? y.w / e.w : 0.f;
  }
  return y;
}

// Float4 words per interior node of the compact operators a launch reads: kwm and kL, and kwe
// while the energy system iterates.
__device__ __forceinline__ double op_words(bool ene) { return 1.25 + (ene ? 1.0 : 0.0); }

// Thread -> interior column (i, j) and its segment [k0, k1) of planes. False for the threads
// past the last column of the plane (they still take part in the block reduction).
struct Column {
  int cb;      // node index of (i, j, 0)
  int k0, k1;  // planes of the segment
};
// A block's index in a two-dimensional grid of (column chunks) x (plane segments), and the grid's
// size: the hardware indices of a launch, or those a persistent kernel assigns.
struct VGrid {
  unsigned x, y, nx, ny;
};
__device__ __forceinline__ VGrid hw_grid() { return {blockIdx.x, blockIdx.y, gridDim.x, gridDim.y}; }

__device__ __forceinline__ bool column(const DevParams& P, Column& col, const VGrid& g) {
  const int N = P.N, ni = N - 2;
  const int q = (int)g.x * blockDim.x + threadIdx.x;
  if (q >= ni * ni) return false;
  const int j = q / ni, i = q - j * ni;
  col.cb = (i + 1) + N * (j + 1);
  col.k0 = 1 + (int)g.y * P.kz;
  col.k1 = min(col.k0 + P.kz, N - 1);
  return true;
}
__device__ __forceinline__ bool column(const DevParams& P, Column& col) {
  return column(P, col, hw_grid());
}

__device__ __forceinline__ unsigned block_id(const VGrid& g) { return g.x + g.nx * g.y; }
__device__ __forceinline__ unsigned block_count(const VGrid& g) { return g.nx * g.ny; }
__device__ __forceinline__ unsigned block_id() { return block_id(hw_grid()); }
__device__ __forceinline__ unsigned block_count() { return block_count(hw_grid()); }

// Per-system scalars of the interleaved kernels, zero for a finished system so that its vectors
// stay as they are (x += 0, r = r - 0).
struct Scal4 {
  float4 a, b, om;
  int done[4];
  int all_done;
};

__device__ __forceinline__ void load_scalars(const KrylovScalars* ks, Scal4& sc) {
  if (threadIdx.x == 0) {
    float a[4], b[4], om[4];
    int all = 1;
    for (int s = 0; s < 4; ++s) {
      const int d = ks[s].done;
      sc.done[s] = d;
      all &= d;
      a[s] = d ? 0.f : (float)ks[s].alpha;
      b[s] = d ? 0.f : (float)ks[s].beta;
      om[s] = d ? 0.f : (float)ks[s].omega;
    }
    sc.a = make_float4(a[0], a[1], a[2], a[3]);
    sc.b = make_float4(b[0], b[1], b[2], b[3]);
    sc.om = make_float4(om[0], om[1], om[2], om[3]);
    sc.all_done = all;
  }
  __syncthreads();
}

// Algorithmic bytes of one interleaved launch: words (float4 per interior node) moved.
__device__ __forceinline__ double bytes4(const DevParams& P, double float4_words) {
  const double ni = (double)(P.N - 2);
  return 16.0 * float4_words * ni * ni * ni;
}

// Programmatic dependent launch: the Krylov kernels of the interleaved solve are launched so that
// each may start while the previous one is finishing (its blocks take SMs as the previous
// kernel's blocks leave); a kernel waits for the previous grid's completion and memory before its
// first access, and lets the next kernel launch at once.
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// r = r_0, x = 0, p = v = 0 at interior nodes, every vector zero on the walls; ||r_0||^2.
// Grid-stride over all N^3 nodes: each thread sums several nodes before the one block reduction.
// Returns true in the block that finished the launch's reduction (its scalars are then final).
__device__ __forceinline__ bool k4_init_body(const DevParams& P, const Fields& F, unsigned vbx,
                                             unsigned vnb) {
  __shared__ double smem[32 * 4];
  const unsigned N = P.N;
  const unsigned n3 = N * N * N;
  FF acc[4] = {};
  for (unsigned c = vbx * blockDim.x + threadIdx.x; c < n3; c += vnb * blockDim.x) {
    const unsigned q = c / N;
    const unsigned i = c - q * N, j = q % N, k = q / N;
    const bool inner = i > 0 && j > 0 && k > 0 && i < N - 1 && j < N - 1 && k < N - 1;
    const float4 z = f4(0.f);
    const float4 r = inner ? F.kr0[c] : z;
    F.kr[c] = r;
    // t needs no zeros: inside, k4_st writes it before k4_xr reads it; its wall entries (and those
    // of r_0) are zero from the workspace's zeroing at creation, and no kernel writes them
    F.kx[c] = z;
    F.kp[0][c] = z;
    F.kp[1][c] = z;
    F.kv[0][c] = z;
    F.kv[1][c] = z;
    ff_dot4(acc, r, r);
  }
  double part[4];
  block_ff<4>(acc, part, smem);
  if (!publish_is_last<4>(part, F.red, F.counter, vbx, vnb)) return false;
  {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, vnb, F.counter, smem);
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
        // an inner pressure pass solves the momentum systems only
        k.done = (k.r0norm == 0.0 || *F.halt || (s == 3 && P.inner_pass)) ? 1 : 0;
      }
    }
  }
  return true;
}

__global__ void __launch_bounds__(kThreads) k4_init(DevParams P, Fields F) {
  k4_init_body(P, F, blockIdx.x, gridDim.x);
}

// p_new = r + beta (p_old - omega v_old) at the seven stencil nodes, v_new = A p_new, partial
// r_0 . v_new; last block: alpha = rho / (r_0 . v_new).
__device__ __forceinline__ void k4_pv_body(const DevParams& P, const Fields& F, int pp,
                                            const VGrid& vg) {
  __shared__ double smem[32 * 4];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return;   // uniform over the grid
  const bool ene = !sc.done[3];   // the energy system still iterates (uniform)
  const int N = P.N, N2 = N * N;
  const float4 b = sc.b, mom = neg4(sc.om);
  const float4* HOSC_RESTRICT R = F.kr;
  const float4* HOSC_RESTRICT Po = F.kp[pp];
  const float4* HOSC_RESTRICT Vo = F.kv[pp];
  float4* HOSC_RESTRICT Pn = F.kp[1 - pp];
  float4* HOSC_RESTRICT Vn = F.kv[1 - pp];
  auto pnew = [&](int c) {
    const float4 r = HOSC_LDG(R + c), p = HOSC_LDG(Po + c), v = HOSC_LDG(Vo + c);
    return fma4(b, fma4(mom, v, p), r);
  };
  FF acc[4] = {};
  Column col;
  if (column(P, col, vg)) {
    float4 pm = pnew(col.cb + N2 * (col.k0 - 1));
    float4 pc = pnew(col.cb + N2 * col.k0);
    for (int k = col.k0; k < col.k1; ++k) {
      const int c = col.cb + N2 * k;
      const float4 pz = pnew(c + N2);
      const float4 vn = apply_op(P, load_op(F, c, ene), pc, pnew(c + 1), pnew(c - 1),
                                 pnew(c + N), pnew(c - N), pz, pm);
      Pn[c] = pc;
      Vn[c] = vn;
      ff_dot4(acc, HOSC_LDG(F.kr0 + c), vn);
      pm = pc;
      pc = pz;
    }
  }
  double part[4];
  block_ff<4>(acc, part, smem);
  if (publish_is_last<4>(part, F.red, F.counter, block_id(vg), block_count(vg))) {
    double tot[4];
    reduce_partials<4, false>(tot, F.red, block_count(vg), F.counter, smem);
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
      // r p v r0 in, p v out, the compact operators
      F.alg_bytes[HOSC_K_BICG_PV] += bytes4(P, 6.0 + op_words(ene));
    }
  }
}

template <int MinB>
__global__ void __launch_bounds__(MinB == 2 ? 384 : 256, MinB)
    k4_pv(DevParams P, Fields F, int pp) {
  pdl_wait_and_release();
  k4_pv_body(P, F, pp, hw_grid());
}

// s = r - alpha v at the seven stencil nodes, t = A s, partials (t . s, t . t); last block:
// omega = (t . s) / (t . t) (0 when t = 0).
__device__ __forceinline__ void k4_st_body(const DevParams& P, const Fields& F, int pp,
                                            const VGrid& vg) {
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return;
  const bool ene = !sc.done[3];   // the energy system still iterates (uniform)
  const int N = P.N, N2 = N * N;
  const int np = 1 - pp;   // written by k4_pv of this iteration
  const float4 ma = neg4(sc.a);
  const float4* HOSC_RESTRICT R = F.kr;
  const float4* HOSC_RESTRICT V = F.kv[np];
  float4* HOSC_RESTRICT T = F.kt;
  auto sval = [&](int c) { return fma4(ma, HOSC_LDG(V + c), HOSC_LDG(R + c)); };
  FF acc[8] = {};
  Column col;
  if (column(P, col, vg)) {
    float4 sm = sval(col.cb + N2 * (col.k0 - 1));
    float4 sc0 = sval(col.cb + N2 * col.k0);
    for (int k = col.k0; k < col.k1; ++k) {
      const int c = col.cb + N2 * k;
      const float4 sz = sval(c + N2);
      const float4 tv = apply_op(P, load_op(F, c, ene), sc0, sval(c + 1), sval(c - 1),
                                 sval(c + N), sval(c - N), sz, sm);
      T[c] = tv;
      ff_dot4(acc, tv, sc0);
      ff_dot4(acc + 4, tv, tv);
      sm = sc0;
      sc0 = sz;
    }
  }
  double part[8];
  block_ff<8>(acc, part, smem);
  if (publish_is_last<8>(part, F.red, F.counter, block_id(vg), block_count(vg))) {
    double tot[8];
    reduce_partials<8, false>(tot, F.red, block_count(vg), F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        k.omega = tot[4 + s] > 0.0 ? tot[s] / tot[4 + s] : 0.0;
      }
      // r v in, t out, the compact operators
      F.alg_bytes[HOSC_K_BICG_ST] += bytes4(P, 3.0 + op_words(ene));
    }
  }
}

template <int MinB>
__global__ void __launch_bounds__(MinB == 2 ? 384 : 256, MinB)
    k4_st(DevParams P, Fields F, int pp) {
  pdl_wait_and_release();
  k4_st_body(P, F, pp, hw_grid());
}

// The last block of an x/r launch: totals of (r_0 . r, r . r) per system, then the convergence and
// breakdown tests, beta and rho of the next iteration.
__device__ __forceinline__ void xr_finish(const DevParams& P, const Fields& F, unsigned nblocks,
                                          double* smem) {
  double tot[8];
  reduce_partials<8, false>(tot, F.red, nblocks, F.counter, smem);
  if (threadIdx.x == 0) {
    for (int s = 0; s < 4; ++s) {
      KrylovScalars& k = F.ks[s];
      if (k.done) continue;
      const double rho_new = tot[s];
      k.rnorm = sqrt(tot[4 + s]);
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
    F.alg_bytes[HOSC_K_BICG_XR] += bytes4(P, 8.0);   // r v p x t r0 in, x r out
  }
}

// s = r - alpha v; x += alpha p + omega s; r = s - omega t; partials (r_0 . r, r . r); last block:
// convergence and breakdown tests, beta and rho of the next iteration.
// Returns true in the block that finished the launch's reduction (convergence decided).
__device__ __forceinline__ bool k4_xr_body(const DevParams& P, const Fields& F, int pp,
                                            const VGrid& vg) {
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  load_scalars(F.ks, sc);
  if (sc.all_done) return false;
  const int N2 = P.N * P.N;
  const int np = 1 - pp;
  const float4 a = sc.a, om = sc.om, ma = neg4(sc.a), mom = neg4(sc.om);
  FF acc[8] = {};
  Column col;
  if (column(P, col, vg)) {
    for (int k = col.k0; k < col.k1; ++k) {
      const int c = col.cb + N2 * k;
      const float4 r = F.kr[c], v = HOSC_LDG(F.kv[np] + c), p = HOSC_LDG(F.kp[np] + c);
      const float4 t = HOSC_LDG(F.kt + c), r0 = HOSC_LDG(F.kr0 + c);
      const float4 sv = fma4(ma, v, r);
      F.kx[c] = fma4(om, sv, fma4(a, p, F.kx[c]));
      const float4 rn = fma4(mom, t, sv);
      F.kr[c] = rn;
      ff_dot4(acc, r0, rn);
      ff_dot4(acc + 4, rn, rn);
    }
  }
  double part[8];
  block_ff<8>(acc, part, smem);
  if (!publish_is_last<8>(part, F.red, F.counter, block_id(vg), block_count(vg))) return false;
  xr_finish(P, F, block_count(vg), smem);
  return true;
}

template <int MinB>
__global__ void __launch_bounds__(MinB == 2 ? 384 : 256, MinB)
    k4_xr(DevParams P, Fields F, int pp) {
  pdl_wait_and_release();
  k4_xr_body(P, F, pp, hw_grid());
}

}  // namespace

}  // namespace hosc
