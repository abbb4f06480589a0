// Device helpers shared by the kernels of libhosc.so: indexing, one-sided / central gradients,
// block reductions and the last-block reduction of per-block partials.
#pragma once

// Loads of arrays that a kernel only reads. A kernel launch reads them through the read-only
// (non-coherent) cache with restrict-qualified pointers. The persistent round kernel of the pool
// (hosc_round.cu, built with HOSC_PERSISTENT_BUILD) writes these arrays in one phase and reads
// them in a later one of the same launch, so there they are plain loads cached in L2 only
// (coherent across SMs), and pointers are not restrict-qualified.
#ifdef HOSC_PERSISTENT_BUILD
#define HOSC_RESTRICT
#define HOSC_LDG(p) __ldcg(p)
#else
#define HOSC_RESTRICT __restrict__
#define HOSC_LDG(p) __ldg(p)
#endif


#include <cuda_runtime.h>

#include "hosc_internal.h"

namespace hosc {

__device__ __forceinline__ long node(int i, int j, int k, int N) {
  return (long)i + (long)N * ((long)j + (long)N * (long)k);
}

// Derivative along one axis at a node whose coordinate along that axis is a (0..N-1); st is the
// memory stride of that axis. Central inside, second-order one-sided at the two walls.
__device__ __forceinline__ double grad_axis(const double* HOSC_RESTRICT f, long c, int a, int N,
                                            long st, double inv2h) {
  if (a == 0) return (-3.0 * f[c] + 4.0 * f[c + st] - f[c + 2 * st]) * inv2h;
  if (a == N - 1) return (3.0 * f[c] - 4.0 * f[c - st] + f[c - 2 * st]) * inv2h;
  return (f[c + st] - f[c - st]) * inv2h;
}

struct Grad9 {
  double ux, uy, uz, vx, vy, vz, wx, wy, wz;
};

// The nine velocity gradients at node (i, j, k); ix, iy, iz = 1/(2 h_d) of the three directions.
__device__ __forceinline__ Grad9 velocity_gradients(const double* HOSC_RESTRICT u,
                                                    const double* HOSC_RESTRICT v,
                                                    const double* HOSC_RESTRICT w, int i, int j,
                                                    int k, int N, double ix, double iy,
                                                    double iz) {
  const long c = node(i, j, k, N);
  const long sy = N, sz = (long)N * N;
  Grad9 g;
  g.ux = grad_axis(u, c, i, N, 1, ix);
  g.uy = grad_axis(u, c, j, N, sy, iy);
  g.uz = grad_axis(u, c, k, N, sz, iz);
  g.vx = grad_axis(v, c, i, N, 1, ix);
  g.vy = grad_axis(v, c, j, N, sy, iy);
  g.vz = grad_axis(v, c, k, N, sz, iz);
  g.wx = grad_axis(w, c, i, N, 1, ix);
  g.wy = grad_axis(w, c, j, N, sy, iy);
  g.wz = grad_axis(w, c, k, N, sz, iz);
  return g;
}

// Second invariant of the strain-rate tensor, Eq. (8).
__device__ __forceinline__ double second_invariant(const Grad9& g) {
  const double a = g.uz + g.wx, b = g.uy + g.vx, c = g.vz + g.wy;
  return 2.0 * (g.ux * g.ux + g.vy * g.vy + g.wz * g.wz) + a * a + b * b + c * c;
}

// ----------------------------------------------------------------------------- reductions

template <int M>
__device__ __forceinline__ void warp_sum(double (&v)[M]) {
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[m] += __shfl_down_sync(0xffffffffu, v[m], off);
}

// Larger of two non-negative doubles (+inf allowed). For such values the IEEE order is the order
// of their bit patterns as integers, so the comparison runs on the integer units: GB300 issues
// FP64 instructions at a small fraction of its integer rate. Every max-reduction here reduces
// magnitudes.
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

template <int M>
__device__ __forceinline__ void warp_max(double (&v)[M]) {
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      v[m] = max_nonneg(v[m], __shfl_down_sync(0xffffffffu, v[m], off));
}

// Sum (or max, of non-negative values) of M values over the block; the result is valid in
// thread 0. Fixed order, so the result is the same run to run for the same launch shape.
// smem: >= 32*M doubles.
template <int M, bool IsMax>
__device__ __forceinline__ void block_reduce(double (&v)[M], double* smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (IsMax) warp_max<M>(v); else warp_sum<M>(v);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) smem[wid * M + m] = v[m];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = (lane < nw) ? smem[lane * M + m] : (IsMax ? 0.0 : 0.0);
    if (IsMax) warp_max<M>(v); else warp_sum<M>(v);
  }
  __syncthreads();
}

// Block sum of M values whose per-thread terms are float: the warp stage adds in float, the
// warp sums are widened to double for the cross-warp stage (and the grid stage that follows), so
// each thread does no double arithmetic. The result is valid in thread 0.
template <int M>
__device__ __forceinline__ void block_sum_f32(const float (&vf)[M], double (&v)[M], double* smem) {
  float w[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    w[m] = vf[m];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w[m] += __shfl_down_sync(0xffffffffu, w[m], off);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) smem[wid * M + m] = (double)w[m];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = (lane < nw) ? smem[lane * M + m] : 0.0;
    warp_sum<M>(v);
  }
  __syncthreads();
}

// Doubles per row of the partials buffer for M values per block: kRedSlots, 2 kRedSlots for
// 8 < M <= 16, 4 kRedSlots for 16 < M <= 32 (one row then spans two or four rows of kRedSlots;
// the kernels with more than 16 values have few enough blocks).
template <int M>
__host__ __device__ constexpr int row_stride() {
  return M > 2 * kRedSlots ? 4 * kRedSlots : (M > kRedSlots ? 2 * kRedSlots : kRedSlots);
}

// Publish the M partials of block b of nb (valid in thread 0) and report whether this block is
// the last one to do so. No thread waits on another block: the last block to take a ticket does
// the final reduction, every other block simply exits.
template <int M>
__device__ __forceinline__ bool publish_is_last(const double (&v)[M], double* red,
                                                unsigned int* counter, unsigned int b,
                                                unsigned int nb) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) red[(long)b * row_stride<M>() + m] = v[m];
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    s_last = (ticket == nb - 1);
  }
  __syncthreads();
  return s_last != 0;
}

// The same for a one-dimensional grid.
template <int M>
__device__ __forceinline__ bool publish_is_last(const double (&v)[M], double* red,
                                                unsigned int* counter) {
  return publish_is_last<M>(v, red, counter, blockIdx.x, gridDim.x);
}

// In the last block: reduce the partials of all blocks in a fixed order (valid in thread 0) and
// re-arm the ticket counter for the next kernel. With Mp the power of two >= M, thread t reads
// slot t % Mp (if below M) of rows t / Mp, t / Mp + blockDim/Mp, ... (consecutive threads read
// consecutive doubles; four rows' loads in flight at a time), then the threads of each slot
// combine through shuffles and shared memory.
// blockDim.x must be a multiple of 32 (and at least Mp); smem: >= 32*M doubles.
template <int M, bool IsMax>
__device__ __forceinline__ void reduce_partials(double (&tot)[M], const double* red, int nblocks,
                                                unsigned int* counter, double* smem) {
  static_assert(M >= 1 && M <= 32, "at most 32 values per block");
  constexpr int Mp = M <= 1 ? 1 : M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 16 ? 16 : 32;
  constexpr long S = row_stride<M>();
  __threadfence();
  const int t = threadIdx.x, bd = blockDim.x;
  const int m = t % Mp, rstep = bd / Mp;
  auto op = [](double a, double b) { return IsMax ? max_nonneg(a, b) : a + b; };
  double acc = 0.0;
  int r = m < M ? t / Mp : nblocks;   // lanes past the M values read nothing
  for (; r + 3 * rstep < nblocks; r += 4 * rstep) {
    const double a0 = __ldcg(red + r * S + m);
    const double a1 = __ldcg(red + (r + rstep) * S + m);
    const double a2 = __ldcg(red + (r + 2 * rstep) * S + m);
    const double a3 = __ldcg(red + (r + 3 * rstep) * S + m);
    acc = op(op(op(op(acc, a0), a1), a2), a3);
  }
  for (; r < nblocks; r += rstep) acc = op(acc, __ldcg(red + r * S + m));
#pragma unroll
  for (int off = 16; off >= Mp; off >>= 1) acc = op(acc, __shfl_down_sync(0xffffffffu, acc, off));
  const int lane = t & 31, wid = t >> 5, nw = bd >> 5;
  if (lane < M) smem[wid * M + lane] = acc;
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < M; ++q) {
      double v = 0.0;
      for (int w = 0; w < nw; ++w) v = op(v, smem[w * M + q]);
      tot[q] = v;
    }
    *counter = 0u;
  }
  __syncthreads();
}

}  // namespace hosc
