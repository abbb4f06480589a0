// Bulk-copy (TMA) stencil kernels of the interleaved FP32 BiCGSTAB (Punia & Ray,
// arXiv:2411.06563, Sec. 2.2: unpreconditioned BiCGSTAB on the four level-(n+1) systems of
// Eq. 5). The p/v and s/t kernels compute what k4_pv and k4_st compute (same operator arithmetic,
// apply_op), with their reads moved by the bulk-copy engine instead of load instructions.
//
// A block owns a tile of ttx * tty interior (i, j) columns and a segment of tkz planes. One
// producer thread (the block's last warp) streams the planes of the segment, S - 2 ahead of the
// plane being computed, into a ring of S shared-memory stages (S = 3, 4, 6 or 8): per plane the haloed
// (ttx + 2) x (tty + 2) box of each stencil vector and the tile boxes of the compact operators
// (and r_0) by tensor-map copies (cp.async.bulk.tensor over 8-byte elements, so that each box row
// is one contiguous run; zero fill outside the grid), and the
// momentum L of each tile row by a plain bulk copy (its rows are not 16-byte aligned in general,
// which a tensor map requires). A stage's copies complete a "full" mbarrier (transaction count);
// the consumer warps mark a stage free on an "empty" mbarrier once they have read it. No load
// instruction of the consumers goes to global memory, so the bytes in flight do not depend on
// registers or resident warps. Every wait is bounded (kTmaWaitNs on the GPU timer): a block whose
// wait runs out marks the four systems done with status HOSC_ECUDA, the producer waits (bounded)
// for the copies it has issued, and the launch ends normally.
#include <cuda.h>
#include <string.h>

#include "hosc_krylov4.cuh"

namespace hosc {

namespace {

constexpr int kTmaMaxThreads = 512;
constexpr unsigned long long kTmaWaitNs = 2000000000ull;   // 2 s
enum { kMapR = 0, kMapR0 = 1, kMapP0 = 2, kMapV0 = 4, kMapWM = 6, kMapWE = 7 };

__host__ __device__ inline int up128(int b) { return (b + 127) & ~127; }

// Byte layout of one stage: the haloed vectors (r, p, v for p/v; r, v for s/t), the momentum
// and energy operator tiles, r_0 (p/v), then one staged row of L per tile row.
struct TmaLayout {
  int tx, ty, lw;    // tile; floats per staged L row
  int nv;            // haloed vectors
  int vb, tb, lrow;  // bytes of a haloed vector box, of a tile box, of a staged L row
  int off_v0, off_m, off_e, off_r0, off_l, stage;
};

__host__ __device__ inline TmaLayout tma_layout(int tx, int ty, bool pv) {
  TmaLayout L;
  L.tx = tx;
  L.ty = ty;
  L.lw = (tx + 3 + 3) & ~3;   // from the 16-byte boundary below column i0 to column i0 + tx - 1
  L.nv = pv ? 3 : 2;
  L.vb = 16 * (tx + 2) * (ty + 2);
  L.tb = 16 * tx * ty;
  L.lrow = 4 * L.lw;
  int off = 0;
  L.off_v0 = off;
  off += L.nv * up128(L.vb);
  L.off_m = off;
  off += up128(L.tb);
  L.off_e = off;
  off += up128(L.tb);
  L.off_r0 = off;
  off += pv ? up128(L.tb) : 0;
  L.off_l = off;
  off += up128(L.lrow * ty);
  L.stage = off;
  return L;
}

__host__ __device__ inline int tma_consumers(int tx, int ty) { return tx * ty; }
__host__ __device__ inline int tma_threads(int tx, int ty) {
  return ((tma_consumers(tx, ty) + 31) / 32 + 1) * 32;   // consumer warps + the producer warp
}
inline size_t tma_smem(int tx, int ty, bool pv, int stages) {
  return (size_t)stages * tma_layout(tx, ty, pv).stage + 128;   // + alignment slack
}

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gpu_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the completion of the barrier's phase of this parity; false after kTmaWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gpu_ns();
  while (!mbar_try(b, parity))
    if (gpu_ns() - t0 > kTmaWaitNs) return false;
  return true;
}
// Tensor-map copy of a 3-D box into shared memory. The float4 arrays are described as
// {2N, N, N} tensors of 8-byte elements (two per node), so that a box row is one contiguous run
// of 16 (tx + 2) bytes and its x coordinate, 2i, is always a 16-byte boundary.
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, int i, int j, int k,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(2 * i), "r"(j), "r"(k), "r"(smem_u32(bar))
      : "memory");
}
// Plain bulk copy: 16-byte aligned source and destination, size a multiple of 16.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------------------ the kernels

// PV: p_new = r + beta (p_old - omega v_old) at the seven stencil nodes, v_new = A p_new, partial
// r_0 . v_new; last block: alpha = rho / (r_0 . v_new).
// !PV: s = r - alpha v at the seven stencil nodes, t = A s, partials (t . s, t . t); last block:
// omega = (t . s) / (t . t).
struct TmaMaps {
  CUtensorMap m[kTmaMaps];
};

template <bool PV, int S>
__global__ void __launch_bounds__(kTmaMaxThreads)
    k7_stencil(DevParams P, Fields F, int pp, const __grid_constant__ TmaMaps tm) {
  constexpr int M = PV ? 4 : 8;
  extern __shared__ unsigned char tdyn[];
  __shared__ double smem[32 * 8];
  __shared__ Scal4 sc;
  __shared__ __align__(8) unsigned long long full[S];
  __shared__ __align__(8) unsigned long long empty[S];
  __shared__ int failed;
  pdl_wait_and_release();
  load_scalars(F.ks, sc);
  if (sc.all_done) return;   // uniform over the grid
  const bool ene = !sc.done[3];
  const int N = P.N, N2 = N * N;
  const TmaLayout L = tma_layout(P.ttx, P.tty, PV);
  const int i0 = 1 + (int)blockIdx.x * L.tx, j0 = 1 + (int)blockIdx.y * L.ty;
  const int k0 = 1 + (int)blockIdx.z * P.tkz, k1 = min(k0 + P.tkz, N - 1);
  const int nplanes = k1 - k0 + 2;   // planes k0 - 1 .. k1
  const int nwc = (tma_consumers(L.tx, L.ty) + 31) >> 5;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = tdyn + ((128u - (smem_u32(tdyn) & 127u)) & 127u);
  const CUtensorMap* maps = tm.m;   // kernel parameters: generic addresses in param space
  const int np = 1 - pp;   // s/t reads the v written by this iteration's p/v
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nwc);
    }
    failed = 0;
    mbar_init_fence();
  }
  __syncthreads();
  FF acc[M] = {};
  if (wid == nwc) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      const CUtensorMap* vm[3];
      vm[0] = maps + kMapR;
      vm[1] = PV ? maps + kMapP0 + pp : maps + kMapV0 + np;
      vm[2] = maps + kMapV0 + pp;
      int rows = 0;   // tile rows inside the grid (the L rows copied)
      for (int t = 0; t < L.ty; ++t) rows += (j0 + t <= N - 2) ? 1 : 0;
      int u = 0;
      for (; u < nplanes; ++u) {
        const int q = k0 - 1 + u, slot = u % S;
        if (u >= S && !mbar_wait(&empty[slot], (unsigned)((u / S - 1) & 1))) break;
        const bool inner = q >= k0 && q < k1;
        unsigned char* st = base + slot * L.stage;
        unsigned bytes = (unsigned)(L.nv * L.vb);
        if (inner)
          bytes += (unsigned)(L.tb + (ene ? L.tb : 0) + (PV ? L.tb : 0) + rows * L.lrow);
        mbar_expect_tx(&full[slot], bytes);
        for (int v = 0; v < L.nv; ++v)
          tma_box(st + L.off_v0 + v * up128(L.vb), vm[v], i0 - 1, j0 - 1, q, &full[slot]);
        if (inner) {
          tma_box(st + L.off_m, maps + kMapWM, i0, j0, q, &full[slot]);
          if (ene) tma_box(st + L.off_e, maps + kMapWE, i0, j0, q, &full[slot]);
          if (PV) tma_box(st + L.off_r0, maps + kMapR0, i0, j0, q, &full[slot]);
          for (int t = 0; t < rows; ++t) {
            const long lin = (long)i0 + (long)N * (j0 + t) + (long)N2 * q;
            bulk_copy(st + L.off_l + t * L.lrow, F.kL + (lin & ~3L), (unsigned)L.lrow,
                      &full[slot]);
          }
        }
      }
      if (u < nplanes) {
        // a wait ran out: wait (bounded) for the copies already issued, the last use of each
        // stage, before the block leaves
        failed = 1;
        for (int s = 0; s < S; ++s) {
          int last = -1;
          for (int w = 0; w < u; ++w)
            if (w % S == s) last = w;
          if (last >= 0) mbar_wait(&full[s], (unsigned)((last / S) & 1));
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- consumers
    const int t = threadIdx.x, tx = t % L.tx, ty = t / L.tx;
    const bool mine = t < L.tx * L.ty && i0 + tx <= N - 2 && j0 + ty <= N - 2;
    const int hx = L.tx + 2;
    const int h = (ty + 1) * hx + (tx + 1), e = ty * L.tx + tx;
    const float4 zero = f4(0.f);
    const float4 b = sc.b, mom = neg4(sc.om), ma = neg4(sc.a);
    auto vec = [&](int u, int v) {
      return (const float4*)(base + (u % S) * L.stage + L.off_v0 + v * up128(L.vb));
    };
    // the stencil vector at haloed index x of the plane of use u
    auto val = [&](int u, int x) {
      if (PV) return fma4(b, fma4(mom, vec(u, 2)[x], vec(u, 1)[x]), vec(u, 0)[x]);
      return fma4(ma, vec(u, 1)[x], vec(u, 0)[x]);
    };
    bool ok = mbar_wait(&full[0], 0u);
    float4 pm = (ok && mine) ? val(0, h) : zero;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[0]);
    ok = ok && mbar_wait(&full[1 % S], (unsigned)((1 / S) & 1));
    float4 pc = (ok && mine) ? val(1, h) : zero;
    for (int u = 1; ok && u < nplanes - 1; ++u) {   // plane k = k0 - 1 + u
      const int un = u + 1;
      if (!mbar_wait(&full[un % S], (unsigned)((un / S) & 1))) {
        ok = false;
        break;
      }
      const float4 pz = mine ? val(un, h) : zero;
      if (mine) {
        const unsigned char* st = base + (u % S) * L.stage;
        const int k = k0 - 1 + u;
        const long lin = (long)i0 + (long)N * (j0 + ty) + (long)N2 * k;
        Op4 op;
        op.m = ((const float4*)(st + L.off_m))[e];
        op.e = ene ? ((const float4*)(st + L.off_e))[e] : zero;
        op.l12 = ((const float*)(st + L.off_l + ty * L.lrow))[(int)(lin & 3L) + tx] *
                 (1.f / 12.f);
        const float4 y = apply_op(P, op, pc, val(u, h + 1), val(u, h - 1), val(u, h + hx),
                                  val(u, h - hx), pz, pm);
        const int c = (i0 + tx) + N * (j0 + ty) + N2 * k;
        if (PV) {
          F.kp[1 - pp][c] = pc;
          F.kv[1 - pp][c] = y;
          ff_dot4(acc, ((const float4*)(st + L.off_r0))[e], y);
        } else {
          F.kt[c] = y;
          ff_dot4(acc, y, pc);
          ff_dot4(acc + 4, y, y);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[u % S]);
      pm = pc;
      pc = pz;
    }
    if (!ok) failed = 1;
  }
  double part[M];
  block_ff<M>(acc, part, smem);   // synchronises the block: failed is final here
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  const bool bad = failed != 0;
  if (publish_is_last<M>(part, F.red, F.counter, bid, nb)) {
    double tot[M];
    reduce_partials<M, false>(tot, F.red, nb, F.counter, smem);
    if (threadIdx.x == 0) {
      for (int s = 0; s < 4; ++s) {
        KrylovScalars& k = F.ks[s];
        if (k.done) continue;
        if (PV) {
          if (tot[s] == 0.0 || !isfinite(tot[s])) {
            k.done = 1;
            k.status = HOSC_ENOCONV;
            continue;
          }
          k.alpha = k.rho / tot[s];
        } else {
          k.omega = tot[4 + s] > 0.0 ? tot[s] / tot[4 + s] : 0.0;
        }
      }
      // p/v: r p v r0 in, p v out; s/t: r v in, t out; the compact operators
      if (PV) F.alg_bytes[HOSC_K_BICG_PV] += bytes4(P, 6.0 + op_words(ene));
      else F.alg_bytes[HOSC_K_BICG_ST] += bytes4(P, 3.0 + op_words(ene));
    }
  }
  if (bad && threadIdx.x == 0) {
    for (int s = 0; s < 4; ++s) {
      F.ks[s].status = HOSC_ECUDA;
      F.ks[s].done = 1;
    }
  }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// A float4 array of N^3 nodes as a 3-D tensor {2N, N, N} of 8-byte elements (the bits are
// copied as they are; outside the tensor the box is filled with zero bits, 0.0f); box
// {2 bw, bh, 1}.
bool encode_vec(CUtensorMap* m, const float4* a, int N, int bw, int bh) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {2ull * N, (cuuint64_t)N, (cuuint64_t)N};
  const cuuint64_t strides[2] = {16ull * N, 16ull * N * N};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * bw), (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)a, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The instantiations: ring depths of 3, 4, 6 and 8 stages (planes 1, 2, 4 and 6 ahead).
template <bool PV>
const void* k7_fn(int stages) {
  switch (stages) {
    case 3: return (const void*)k7_stencil<PV, 3>;
    case 4: return (const void*)k7_stencil<PV, 4>;
    case 6: return (const void*)k7_stencil<PV, 6>;
    case 8: return (const void*)k7_stencil<PV, 8>;
    default: return nullptr;
  }
}

bool tma_attrs_ready() {
  static int done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (!done[dev]) {
    const int cap = 200 * 1024;
    for (int st : {3, 4, 6, 8}) {
      if (cudaFuncSetAttribute(k7_fn<true>(st), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               cap) != cudaSuccess ||
          cudaFuncSetAttribute(k7_fn<false>(st), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
    }
    done[dev] = 1;
  }
  return true;
}

dim3 tma_grid(const DevParams& P) {
  const int ni = P.N - 2;
  return dim3((ni + P.ttx - 1) / P.ttx, (ni + P.tty - 1) / P.tty, (ni + P.tkz - 1) / P.tkz);
}

template <bool PV, int S>
void launch_k7(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = tma_grid(P);
  cfg.blockDim = dim3(tma_threads(P.ttx, P.tty));
  cfg.dynamicSmemBytes = tma_smem(P.ttx, P.tty, PV, S);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TmaMaps tm;
  memcpy(&tm, F.tmaps_host, sizeof(tm));
  cudaLaunchKernelEx(&cfg, k7_stencil<PV, S>, P, F, pp, tm);
}

template <bool PV>
void launch_k7(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  switch (P.tstages) {
    case 4: launch_k7<PV, 4>(P, F, pp, s); break;
    case 6: launch_k7<PV, 6>(P, F, pp, s); break;
    case 8: launch_k7<PV, 8>(P, F, pp, s); break;
    default: launch_k7<PV, 3>(P, F, pp, s); break;
  }
}

}  // namespace

int tma_tile_x(int N) {
  const int ni = N - 2;
  // whole rows up to 126 columns: a haloed row is 2 (tx + 2) <= 256 elements of a box dimension
  const int parts = (ni + 125) / 126;
  return (ni + parts - 1) / parts;
}

bool tma_tiles_valid(int N, int tty, int tkz, int stages) {
  const int ni = N - 2, tx = tma_tile_x(N);
  if (tty < 1 || tty > ni || tkz < 1 || tkz > ni) return false;
  if (stages != 3 && stages != 4 && stages != 6 && stages != 8) return false;
  if (tma_threads(tx, tty) > kTmaMaxThreads) return false;
  if (tma_smem(tx, tty, true, stages) > 200 * 1024) return false;
  if (tty + 2 > 256) return false;
  const long nb = (long)((ni + tx - 1) / tx) * ((ni + tty - 1) / tty) * ((ni + tkz - 1) / tkz);
  const long n3 = (long)N * N * N;
  return nb <= red_rows(n3) && (ni + tkz - 1) / tkz <= 65535 && (ni + tty - 1) / tty <= 65535;
}

long tma_blocks(const DevParams& P) {
  if (P.tty <= 0) return 0;
  const dim3 g = tma_grid(P);
  return (long)g.x * g.y * g.z;
}

bool tma_prepare(const DevParams& P, const Fields& F, void* host) {
  if (P.tty <= 0) return true;
  if (!tma_attrs_ready()) return false;
  CUtensorMap* m = (CUtensorMap*)host;
  static_assert(sizeof(CUtensorMap) == kTmaMapBytes, "tensor map size");
  const int tx = P.ttx, ty = P.tty, N = P.N;
  bool ok = encode_vec(m + kMapR, F.kr, N, tx + 2, ty + 2) &&
            encode_vec(m + kMapR0, F.kr0, N, tx, ty) &&
            encode_vec(m + kMapP0, F.kp[0], N, tx + 2, ty + 2) &&
            encode_vec(m + kMapP0 + 1, F.kp[1], N, tx + 2, ty + 2) &&
            encode_vec(m + kMapV0, F.kv[0], N, tx + 2, ty + 2) &&
            encode_vec(m + kMapV0 + 1, F.kv[1], N, tx + 2, ty + 2) &&
            encode_vec(m + kMapWM, F.kwm, N, tx, ty) && encode_vec(m + kMapWE, F.kwe, N, tx, ty);
  return ok;
}

double tma_wave_cost(int N, int tty, int tkz, int stages, int sms) {
  if (!tma_tiles_valid(N, tty, tkz, stages) || !tma_attrs_ready()) return 1e300;
  const int tx = tma_tile_x(N), ni = N - 2;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k7_fn<true>(stages),
                                                    tma_threads(tx, tty),
                                                    tma_smem(tx, tty, true, stages)) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return 1e300;
  }
  const long items = (long)((ni + tx - 1) / tx) * ((ni + tty - 1) / tty) * ((ni + tkz - 1) / tkz);
  const long slots = (long)occ * sms;
  const long waves = (items + slots - 1) / slots;
  // a block streams tkz + 2 planes, stages - 2 of them ahead of the one it computes
  return (double)waves * (tkz + 2) / (double)(stages - 2);
}

void launch_tma_pv(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  launch_k7<true>(P, F, pp, s);
}

void launch_tma_st(const DevParams& P, const Fields& F, int pp, cudaStream_t s) {
  launch_k7<false>(P, F, pp, s);
}

}  // namespace hosc
