// The persistent round kernel of the pool: one launch advances every member cavity of a pool by
// a round of G pseudo-time steps (Punia & Ray, arXiv:2411.06563, Sec. 2.2 solution procedure,
// for many cavities of different sizes at once).
//
// The grid is cooperative (every block resident). Each member advances through the phases of its
// own steps (S1, S2, S3/S4, the Krylov initialisation, the p/v, s/t and x/r kernels of each
// BiCGSTAB iteration, the update kernels, the record, the float copies); a phase's work is a list
// of tiles (the 256-thread blocks of the per-kernel launches), appended to a queue shared by all
// members when the member's previous phase completes, and any block takes the next tile of the
// queue, whatever member it belongs to. The tiles run the same device bodies as the per-kernel
// launches (hosc_step_dev.cuh, hosc_krylov4.cuh) with the member's parameters and arrays; each
// member's reductions finish in its own last tile (its ticket counter, as in the per-kernel
// path), and the block that finishes the last outstanding tile of a phase decides and queues the
// member's next phase (the BiCGSTAB loop continues while one of its systems has not converged).
// No block waits for a particular other block.
//
// Every wait is bounded: a block that waits for a queue position longer than kBarrierNs gives up,
// raises the round's error flag and returns, and so does every other block at its next wait. The
// host reports HOSC_ECUDA for such a round.

#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <vector>

// Arrays written in one phase are read in a later one of the same launch: no read-only-cache
// loads and no restrict-qualified pointers in the device bodies (hosc_device.cuh), and this
// translation unit is built with global loads cached in L2 only.
#define HOSC_PERSISTENT_BUILD 1
#include "hosc_krylov4.cuh"
#include "hosc_step_dev.cuh"

namespace hosc {

namespace {

constexpr unsigned long long kBarrierNs = 5000000000ull;   // 5 s
constexpr int kRoundThreads = 256;
constexpr int kRoundMinBlocks = 4;   // resident blocks per SM the register budget is set for

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void shadow_item(const RoundMember& M, int lev, int tile) {
  const DevParams& P = M.P;
  const Fields& F = M.F;
  const int n3 = P.N * P.N * P.N;
  k_shadow_body(n3, F.u[lev], F.v[lev], F.w[lev], F.th, F.p, F.us[lev], F.vs[lev], F.ws[lev],
                F.ths, F.ps, F.halt, (unsigned)tile);
}

__device__ __noinline__ void rhs_float_item(const RoundMember& M, int cur, int tile) {
  const DevParams& P = M.P;
  const Fields& F = M.F;
  const int o = 1 - cur;
  auto T = [](double* p) { return reinterpret_cast<const float*>(p); };
  k_rhs_body<float, float>(P, F.us[cur], F.vs[cur], F.ws[cur], F.ths, T(F.L[cur]), T(F.Eu[cur]),
                           T(F.Ev[cur]), T(F.Ew[cur]), T(F.L[o]), F.us[o], F.vs[o], F.ws[o],
                           T(F.Eu[o]), T(F.Ev[o]), T(F.Ew[o]), F, (unsigned)tile);
}

// FP64 defect sweeps: the right-hand side in double, stored for the FP32 solve
__device__ __noinline__ void rhs_double_item(const RoundMember& M, int cur, int tile) {
  const DevParams& P = M.P;
  const Fields& F = M.F;
  const int o = 1 - cur;
  k_rhs_body<double, float>(P, F.u[cur], F.v[cur], F.w[cur], F.th, F.L[cur], F.Eu[cur], F.Ev[cur],
                            F.Ew[cur], F.L[o], F.u[o], F.v[o], F.w[o], F.Eu[o], F.Ev[o], F.Ew[o],
                            F, (unsigned)tile);
}

__device__ __forceinline__ void rhs_item(const RoundMember& M, int cur, int tile) {
  if (M.P.sweep_fp32) rhs_float_item(M, cur, tile);
  else rhs_double_item(M, cur, tile);
}

__device__ __forceinline__ VGrid krylov_grid(const RoundMember& M, int tile) {
  VGrid g;
  g.nx = (unsigned)M.kx;
  g.ny = (unsigned)M.ky;
  g.y = (unsigned)tile / g.nx;
  g.x = (unsigned)tile - g.y * g.nx;
  return g;
}

// Each phase's item is a function of its own (not inlined), so that the register allocation of
// one phase (the double right-hand side needs the most) does not spill in the others.
__device__ __noinline__ void visc_item(const RoundMember& M, int cur, int tile) {
  const DevParams& P = M.P;
  const Fields& F = M.F;
  if (P.sweep_fp32)
    k_viscosity_body<float>(P, F.us[cur], F.vs[cur], F.ws[cur], reinterpret_cast<float*>(F.eta),
                            reinterpret_cast<float*>(F.L[cur]), F.halt, (unsigned)tile);
  else
    k_viscosity_body<double>(P, F.u[cur], F.v[cur], F.w[cur], F.eta, F.L[cur], F.halt,
                             (unsigned)tile);
}

__device__ __noinline__ void sources_item(const RoundMember& M, int cur, int tile) {
  const DevParams& P = M.P;
  const Fields& F = M.F;
  if (P.sweep_fp32)
    k_sources_body<float>(P, F.us[cur], F.vs[cur], F.ws[cur], F.ths, F.ps,
                          reinterpret_cast<const float*>(F.eta),
                          reinterpret_cast<float*>(F.Eu[cur]),
                          reinterpret_cast<float*>(F.Ev[cur]), reinterpret_cast<float*>(F.Ew[cur]),
                          F.halt, (unsigned)tile);
  else
    k_sources_body<double>(P, F.u[cur], F.v[cur], F.w[cur], F.th, F.p, F.eta, F.Eu[cur],
                           F.Ev[cur], F.Ew[cur], F.halt, (unsigned)tile);
}

__device__ __noinline__ bool init_item(const RoundMember& M, int tile) {
  return k4_init_body(M.P, M.F, (unsigned)tile, (unsigned)M.init);
}
__device__ __noinline__ void pv_item(const RoundMember& M, int pp, int tile) {
  k4_pv_body(M.P, M.F, pp, krylov_grid(M, tile));
}
__device__ __noinline__ void st_item(const RoundMember& M, int pp, int tile) {
  k4_st_body(M.P, M.F, pp, krylov_grid(M, tile));
}
__device__ __noinline__ bool xr_item(const RoundMember& M, int pp, int tile) {
  return k4_xr_body(M.P, M.F, pp, krylov_grid(M, tile));
}
__device__ __noinline__ void update_item(const RoundMember& M, int phase, int cur, int tile) {
  switch (phase) {
    case 0: k_apply_increment_body<float>(M.P, M.F, cur, M.nodes, (unsigned)tile); break;
    case 1: k_theta_walls_body(M.P, M.F, M.theta_walls, (unsigned)tile); break;
    case 2: k_divergence_body(M.P, M.F, 1 - cur, M.interior, (unsigned)tile); break;
    case 3: k_pressure_correct_body(M.P, M.F, (unsigned)tile); break;
    case 4: k_pressure_walls_body(M.P, M.F, (unsigned)tile); break;
    default: k_finish_record_body(M.P, M.F, (unsigned)tile); break;
  }
}

// ------------------------------------------------------------ the work-list (dataflow) form
//
// Each member advances through the phases of its own steps; no block waits for all the others.
// The items of a member's phase are appended to a shared queue when the member's previous phase
// completes: the block that finishes the last outstanding tile of a phase (a per-member counter)
// decides the next phase (the BiCGSTAB loop continues while one of the member's systems has not
// converged) and appends its tiles. Blocks claim queue positions in order; a position is ready
// when its sequence number has been written. A block waits (bounded) only for the next position
// to be filled or for every member to finish the round.

enum FlowPhase {
  PH_SHADOW0 = 0, PH_VISC, PH_SOURCES, PH_RHS, PH_INIT, PH_PV, PH_ST, PH_XR, PH_INC, PH_TWALLS,
  PH_DIV, PH_PCORR, PH_PWALLS, PH_FINISH, PH_SHADOW, PH_DONE
};

struct FlowMember {
  int step;      // steps done in this round
  int it;        // BiCGSTAB iteration of the current step
  int phase;     // current phase
  int pending;   // tiles of the current phase not finished
};

struct FlowDev {
  const RoundMember* m;
  FlowMember* st;
  int count, G, max_it;
  int2* items;          // [cap]: (member, phase << 24 | tile)
  unsigned* seq;        // [cap]: queue position + 1 once the item at that position is written
  unsigned cap;         // a power of two
  unsigned* head;       // next position to claim
  unsigned* tail;       // next position to fill
  int* remaining;       // members still running in this round
  int* err;
};

__device__ __forceinline__ int flow_tiles(const RoundMember& M, int ph) {
  switch (ph) {
    case PH_RHS: case PH_DIV: case PH_PCORR: return M.interior;
    case PH_INIT: return M.init;
    case PH_PV: case PH_ST: case PH_XR: return M.kx * M.ky;
    case PH_TWALLS: return M.theta_walls;
    case PH_PWALLS: return M.pressure_walls;
    case PH_FINISH: return 1;
    default: return M.nodes;   // shadows, viscosity, sources, increments
  }
}

__device__ __forceinline__ void flow_item(const RoundMember& M, int step, int it, int ph,
                                          int tile) {
  const int cur = M.cur ^ (step & 1);
  switch (ph) {
    case PH_SHADOW0: shadow_item(M, M.cur, tile); break;
    case PH_VISC: visc_item(M, cur, tile); break;
    case PH_SOURCES: sources_item(M, cur, tile); break;
    case PH_RHS: rhs_item(M, cur, tile); break;
    case PH_INIT: init_item(M, tile); break;
    case PH_PV: pv_item(M, it & 1, tile); break;
    case PH_ST: st_item(M, it & 1, tile); break;
    case PH_XR: xr_item(M, it & 1, tile); break;
    case PH_SHADOW: shadow_item(M, 1 - cur, tile); break;
    default: update_item(M, ph - PH_INC, cur, tile); break;   // PH_INC .. PH_FINISH
  }
}

__device__ __forceinline__ bool any_active(const RoundMember& M) {
  const volatile KrylovScalars* ks = M.F.ks;
  return !(ks[0].done && ks[1].done && ks[2].done && ks[3].done);
}

// The phase after ph completed (thread 0 of the completing block); PH_DONE ends the round.
__device__ int flow_next(const FlowDev& D, int mb, int ph) {
  const RoundMember& M = D.m[mb];
  FlowMember& S = D.st[mb];
  switch (ph) {
    case PH_INIT:
      S.it = 0;
      return any_active(M) ? PH_PV : PH_INC;
    case PH_XR:
      S.it += 1;
      return (any_active(M) && S.it <= D.max_it) ? PH_PV : PH_INC;
    case PH_FINISH: return *(volatile int*)M.F.halt ? PH_DONE : PH_SHADOW;
    case PH_SHADOW:
      S.step += 1;
      return S.step >= D.G ? PH_DONE : PH_VISC;
    default: return ph + 1;
  }
}

// Start member mb's phase ph: its tile count, then its items at the end of the queue (the whole
// block writes them; s_base is shared scratch).
__device__ void flow_start(const FlowDev& D, int mb, int ph, unsigned* s_base, int* s_n) {
  if (threadIdx.x == 0) {
    if (ph == PH_DONE) {
      *s_n = 0;
      atomicSub(D.remaining, 1);
    } else {
      const int n = flow_tiles(D.m[mb], ph);
      D.st[mb].phase = ph;
      D.st[mb].pending = n;
      *s_n = n;
      *s_base = atomicAdd(D.tail, (unsigned)n);
    }
  }
  __syncthreads();
  const int n = *s_n;
  const unsigned base = *s_base;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    D.items[(base + k) & (D.cap - 1)] = make_int2(mb, (ph << 24) | k);
  __threadfence();
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    atomicExch(D.seq + ((base + k) & (D.cap - 1)), base + k + 1u);
  __syncthreads();
}

__global__ void __launch_bounds__(kRoundThreads, kRoundMinBlocks) k_flow(FlowDev D) {
  __shared__ int s_exit, s_mb, s_ph, s_tile, s_last, s_n, s_step, s_it;
  __shared__ unsigned s_base;
  // the round's start: arm each member (run, stop at its first steady step, no records yet) and
  // queue its first phase
  for (int mb = blockIdx.x; mb < D.count; mb += gridDim.x) {
    const RoundMember& M = D.m[mb];
    if (threadIdx.x == 0) {
      *M.F.halt = 0;
      *M.F.ring_pos = 0u;
      *M.F.steady_stop = 1;
      D.st[mb].step = 0;
      D.st[mb].it = 0;
    }
    flow_start(D, mb, M.P.sweep_fp32 ? PH_SHADOW0 : PH_VISC, &s_base, &s_n);
  }
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned pos = atomicAdd(D.head, 1u);
      const unsigned slot = pos & (D.cap - 1);
      const unsigned long long t0 = now_ns();
      s_exit = 0;
      for (;;) {
        if (*(volatile unsigned*)(D.seq + slot) == pos + 1u) {
          __threadfence();
          const int2 it = __ldcg(D.items + slot);
          s_mb = it.x;
          s_ph = it.y >> 24;
          s_tile = it.y & 0xffffff;
          s_step = __ldcg(&D.st[it.x].step);
          s_it = __ldcg(&D.st[it.x].it);
          break;
        }
        if (*(volatile int*)D.remaining <= 0 || *(volatile int*)D.err) {
          s_exit = 1;
          break;
        }
        if (now_ns() - t0 > kBarrierNs) {
          atomicExch(D.err, 1);
          s_exit = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __syncthreads();
    if (s_exit) return;
    const int mb = s_mb, ph = s_ph;
    flow_item(D.m[mb], s_step, s_it, ph, s_tile);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicSub(&D.st[mb].pending, 1) == 1;
      if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) {
      if (threadIdx.x == 0) s_ph = flow_next(D, mb, ph);
      __syncthreads();
      flow_start(D, mb, s_ph, &s_base, &s_n);
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------------------ host

struct RoundState {
  int device = -1;
  int capacity = 0;       // members the device arrays hold
  RoundMember* d_m = nullptr;
  FlowMember* d_st = nullptr;
  int2* d_items = nullptr;
  unsigned* d_seq = nullptr;
  unsigned* d_ctl = nullptr;   // head, tail, remaining, err
  int flow_grid = 0;
};

constexpr unsigned kQueueCap = 1u << 18;   // queue positions (items of all members in flight)

RoundState* round_state_create() { return new RoundState(); }

void round_state_destroy(RoundState* S) {
  if (!S) return;
  if (S->d_m) cudaFree(S->d_m);
  if (S->d_st) cudaFree(S->d_st);
  if (S->d_items) cudaFree(S->d_items);
  if (S->d_seq) cudaFree(S->d_seq);
  if (S->d_ctl) cudaFree(S->d_ctl);
  delete S;
}

void round_member_shape(RoundMember* M) {
  const long N = M->P.N, n3 = N * N * N, ni = N - 2;
  M->nodes = red_blocks(n3);
  M->interior = red_blocks(ni * ni * ni);
  M->theta_walls = red_blocks(2 * ni * N + 2 * ni * ni);
  M->pressure_walls = red_blocks(n3 - ni * ni * ni);
  M->P.kblock = kRoundThreads;
  M->P.kz = (int)(ni < 8 ? ni : 8);
  M->P.narrow = 0;
  M->P.merged = 0;
  M->P.sx = M->P.sy = M->P.skz = 0;
  // the Krylov initialisation strides over the nodes with at most one wave of blocks, as its
  // own launch does (same partial sums, same reduction order)
  const int most = 8 * device_sms();
  M->init = M->nodes < most ? M->nodes : most;
  M->kx = (int)((ni * ni + kRoundThreads - 1) / kRoundThreads);
  M->ky = (int)((ni + M->P.kz - 1) / M->P.kz);
}

hosc_status launch_flow(RoundState* S, const std::vector<RoundMember>& members, int G,
                        cudaStream_t stream, char* detail, size_t detail_len) {
  const int count = (int)members.size();
  if (count == 0) return HOSC_OK;
  int max_it = 1;
  for (const RoundMember& M : members)
    max_it = M.P.max_lin_iter > max_it ? M.P.max_lin_iter : max_it;
  auto fail = [&](const char* what, cudaError_t e) {
    snprintf(detail, detail_len, "round kernel: %s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return HOSC_ECUDA;
  };
  // the tiles of one phase of every member must fit in the queue at once
  long most = 0;
  for (const RoundMember& M : members) {
    long m = M.nodes;
    if (M.interior > m) m = M.interior;
    if ((long)M.kx * M.ky > m) m = (long)M.kx * M.ky;
    most += m;
  }
  cudaError_t e = cudaSuccess;
  int device = 0;
  if ((e = cudaGetDevice(&device)) != cudaSuccess) return fail("device", e);
  if (most + 4096 > (long)kQueueCap) {
    snprintf(detail, detail_len, "round kernel: %ld tiles in one phase exceed the queue (%u)",
             most, kQueueCap);
    return HOSC_ENOMEM;
  }
  if (S->device != device || S->capacity < count || !S->d_st) {
    if (S->d_m) cudaFree(S->d_m);
    if (S->d_st) cudaFree(S->d_st);
    if (S->d_items) cudaFree(S->d_items);
    if (S->d_seq) cudaFree(S->d_seq);
    if (S->d_ctl) cudaFree(S->d_ctl);
    S->d_m = nullptr;
    S->d_st = nullptr;
    S->d_items = nullptr;
    S->d_seq = nullptr;
    S->d_ctl = nullptr;
    const int cap = count < 16 ? 16 : count * 2;
    if ((e = cudaMalloc(&S->d_m, cap * sizeof(RoundMember))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_st, cap * sizeof(FlowMember))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_items, kQueueCap * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_seq, kQueueCap * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&S->d_ctl, 4 * sizeof(unsigned))) != cudaSuccess) {
      S->capacity = 0;
      return fail("allocation", e);
    }
    S->capacity = cap;
    S->device = device;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_flow, kRoundThreads, 0)) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
      return fail("occupancy", e);
    if (per_sm < 1) return fail("occupancy", cudaErrorInvalidConfiguration);
    S->flow_grid = per_sm * sms;
  }
  const unsigned ctl[4] = {0u, 0u, (unsigned)count, 0u};
  if ((e = cudaMemcpyAsync(S->d_m, members.data(), count * sizeof(RoundMember),
                           cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(S->d_seq, 0, kQueueCap * sizeof(unsigned), stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(S->d_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, stream)) !=
          cudaSuccess)
    return fail("table", e);
  FlowDev D;
  D.m = S->d_m;
  D.st = S->d_st;
  D.count = count;
  D.G = G;
  D.max_it = max_it;
  D.items = S->d_items;
  D.seq = S->d_seq;
  D.cap = kQueueCap;
  D.head = S->d_ctl;
  D.tail = S->d_ctl + 1;
  D.remaining = (int*)(S->d_ctl + 2);
  D.err = (int*)(S->d_ctl + 3);
  void* args[] = {&D};
  if ((e = cudaLaunchCooperativeKernel((const void*)k_flow, dim3(S->flow_grid),
                                       dim3(kRoundThreads), args, 0, stream)) != cudaSuccess)
    return fail("launch", e);
  unsigned back[4] = {0u, 0u, 0u, 0u};
  if ((e = cudaMemcpyAsync(back, S->d_ctl, sizeof(back), cudaMemcpyDeviceToHost, stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return fail("run", e);
  if (back[3]) {
    snprintf(detail, detail_len, "round kernel: a queue wait gave up after %.0f s",
             kBarrierNs * 1e-9);
    return HOSC_ECUDA;
  }
  return HOSC_OK;
}

}  // namespace hosc
