// A pool of cavity solves that advance together on one GPU: the batching and serving layer above
// the single-cavity contexts of hosc_api.cu (declared in include/hosc.h).
//
// Members are contexts (one cavity each, any N, Ra, n) admitted against a device-memory budget.
// hosc_pool_run advances every active member by rounds of G captured steps (each step with its
// BiCGSTAB loop as a device-side WHILE node, each member stopping on the device at its first
// steady step), then folds the step records on the host and completes the members that are
// steady, failed or out of steps. Two ways to issue a round:
//   streams: every member launches its own captured steps on its own stream;
//   graph:   one captured graph holds the round of every member, forked into one branch per
//            member, so a whole round of all cavities is a single graph launch. It is captured
//            again only when the membership or a member's level parity, history, phase or
//            launch shape changes.
//   persistent: one launch of the persistent round kernel (hosc_round.cu) runs the round of
//            every member: its blocks walk each phase's (member, tile) work list.
// The first member of each N that completes a round tunes the launch shape of the mixed
// precision solve (hosc_autotune); later members of that N reuse it.

#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <array>
#include <chrono>
#include <map>
#include <new>
#include <vector>

#include "hosc.h"
#include "hosc_internal.h"

using namespace hosc;

namespace {

#define PCU(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      snprintf(detail_buffer(), 256, "%s: %s", #call, cudaGetErrorString(e_));      \
      return HOSC_ECUDA;                                                            \
    }                                                                               \
  } while (0)

enum { kFree = 0, kActive = 1, kDone = 2 };

struct Member {
  void* ctx = nullptr;
  int state = kFree;
  int N = 0;
  size_t bytes = 0;
  long max_steps = 0;
  hosc_status status = HOSC_OK;
  hosc_info info = {};
  hosc_diag diag = {};
  long signature = -1;    // ctx_signature when the pool graph was captured
  cudaEvent_t join = nullptr;
};

struct Pool {
  size_t budget = 0, used = 0;
  int G = 8;
  int mode = HOSC_POOL_STREAMS;
  int autotune = 1;
  int device = 0;
  std::vector<Member> m;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;                          // membership changed since the capture
  // tuned launch shapes per N: kblock, kz, narrow, sx, sy, skz, tty, tkz, merged, x/r form,
  // ring stages and kernels of the bulk-copy kernels
  std::map<int, std::array<int, 12>> tiles;
  long rounds = 0, captures = 0;
  double capture_ms = 0.0;
  RoundState* rs = nullptr;                   // persistent mode: the round kernel's tables
};

void drop_exec(Pool* P) {
  if (P->exec) {
    cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
  }
}

// One graph for the round of every active member: fork one branch per member from the pool's
// stream, append the member's round on it, join.
hosc_status capture_round(Pool* P) {
  const auto t0 = std::chrono::steady_clock::now();
  drop_exec(P);
  PCU(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
  hosc_status st = HOSC_OK;
  cudaError_t e = cudaEventRecord(P->fork, P->stream);
  for (Member& q : P->m) {
    if (q.state != kActive || e != cudaSuccess || st) continue;
    cudaStream_t b = ctx_branch_stream(q.ctx);
    e = cudaStreamWaitEvent(b, P->fork, 0);
    if (e == cudaSuccess) st = ctx_append_round(q.ctx, P->G);
    if (e == cudaSuccess && !st) e = cudaEventRecord(q.join, b);
    if (e == cudaSuccess && !st) e = cudaStreamWaitEvent(P->stream, q.join, 0);
    q.signature = ctx_signature(q.ctx);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(P->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && !st) e = cudaGraphInstantiate(&P->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (st) return st;
  if (e != cudaSuccess) {
    snprintf(detail_buffer(), 256, "pool round capture: %s", cudaGetErrorString(e));
    return HOSC_ECUDA;
  }
  P->dirty = false;
  P->captures += 1;
  P->capture_ms +=
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return HOSC_OK;
}

bool needs_capture(const Pool* P) {
  if (P->dirty || !P->exec) return true;
  for (const Member& q : P->m)
    if (q.state == kActive && q.signature != ctx_signature(q.ctx)) return true;
  return false;
}

hosc_status apply_shape(void* ctx, const std::array<int, 12>& t) {
  hosc_status st = hosc_set_krylov_merged(ctx, t[8]);
  if (!st) st = hosc_set_tiles(ctx, t[0], t[1], t[2]);
  if (!st) st = hosc_set_stencil_tiles(ctx, t[3], t[4], t[5]);
  if (!st) st = hosc_set_tma_tiles(ctx, t[6], t[7], t[10], t[11]);
  if (!st) st = hosc_set_xr_form(ctx, t[9]);
  return st;
}

// After a member's round: complete it (steady, failed, out of steps) or tune its launch shape.
hosc_status settle(Pool* P, int slot, hosc_status st, bool steady, const hosc_info& ri,
                   int* done, int cap, int* ndone) {
  Member& q = P->m[slot];
  q.info.steps += ri.steps;
  q.info.lin_iters += ri.lin_iters;
  q.info.solve_iters += ri.solve_iters;
  for (int s = 0; s < 4; ++s) q.info.sys_iters[s] += ri.sys_iters[s];
  for (int s = 0; s < 4; ++s) q.info.last_iters[s] = ri.last_iters[s];
  if (ri.steps > 0) {
    q.info.res_steady = ri.res_steady;
    q.info.div_max = ri.div_max;
    q.info.lin_res = ri.lin_res;
  }
  q.info.status = ri.status;
  hosc_status fin = HOSC_OK;
  bool complete = false;
  if (st) {
    fin = st;
    complete = true;
  } else if (steady) {
    complete = true;
  } else if (q.info.steps >= q.max_steps) {
    fin = HOSC_ESTEPLIMIT;
    complete = true;
  }
  if (complete) {
    q.state = kDone;
    q.status = fin;
    P->dirty = true;
    if (fin == HOSC_OK || fin == HOSC_ESTEPLIMIT) {
      hosc_status ds = hosc_diagnostics(q.ctx, &q.diag, nullptr, nullptr);
      if (ds) return ds;
    }
    if (*ndone < cap && done) done[*ndone] = slot;
    *ndone += 1;
    return HOSC_OK;
  }
  if (P->autotune && P->mode != HOSC_POOL_PERSISTENT) {
    hosc_params prm;
    if (hosc_get_params(q.ctx, &prm) == HOSC_OK && prm.precision == HOSC_MIXED) {
      auto it = P->tiles.find(q.N);
      if (it == P->tiles.end()) {
        hosc_status ts = hosc_autotune(q.ctx, 3, nullptr, nullptr, nullptr);
        std::array<int, 12> t = {};
        if (!ts) ts = hosc_get_tiles(q.ctx, &t[0], &t[1], &t[2]);
        if (!ts) ts = hosc_get_stencil_tiles(q.ctx, &t[3], &t[4], &t[5]);
        if (!ts) ts = hosc_get_tma_tiles(q.ctx, &t[6], &t[7], &t[10], &t[11]);
        if (!ts) t[8] = hosc_get_krylov_merged(q.ctx);
        if (!ts) t[9] = hosc_get_xr_form(q.ctx);
        if (ts) return ts;
        P->tiles[q.N] = t;
      } else {
        hosc_status ts = apply_shape(q.ctx, it->second);
        if (ts) return ts;
      }
    }
  }
  return HOSC_OK;
}

}  // namespace

extern "C" {

hosc_status hosc_pool_create(size_t budget_bytes, int steps_per_round, int mode, int autotune,
                             void** pool) {
  if (!pool) return HOSC_EINVAL;
  *pool = nullptr;
  if (budget_bytes == 0 || steps_per_round < 1 || steps_per_round > 256) return HOSC_EINVAL;
  if (mode != HOSC_POOL_STREAMS && mode != HOSC_POOL_GRAPH && mode != HOSC_POOL_PERSISTENT)
    return HOSC_EINVAL;
  if (mode == HOSC_POOL_GRAPH && steps_per_round % 2 != 0) return HOSC_EINVAL;
  Pool* P = new (std::nothrow) Pool();
  if (!P) return HOSC_ENOMEM;
  P->budget = budget_bytes;
  P->G = steps_per_round;
  P->mode = mode;
  P->autotune = autotune ? 1 : 0;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
  if (e == cudaSuccess && mode == HOSC_POOL_PERSISTENT) {
    P->rs = round_state_create();
    if (!P->rs) {
      hosc_pool_destroy(P);
      return HOSC_ENOMEM;
    }
  }
  if (e != cudaSuccess) {
    snprintf(detail_buffer(), 256, "pool create: %s", cudaGetErrorString(e));
    hosc_pool_destroy(P);
    return HOSC_ECUDA;
  }
  *pool = P;
  return HOSC_OK;
}

void hosc_pool_destroy(void* pool) {
  Pool* P = (Pool*)pool;
  if (!P) return;
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  drop_exec(P);
  for (Member& q : P->m) {
    if (q.ctx) hosc_destroy(q.ctx);
    if (q.join) cudaEventDestroy(q.join);
  }
  if (P->fork) cudaEventDestroy(P->fork);
  if (P->stream) cudaStreamDestroy(P->stream);
  round_state_destroy(P->rs);
  delete P;
}

hosc_status hosc_pool_admit(void* pool, const hosc_params* params, long max_steps, int* slot) {
  Pool* P = (Pool*)pool;
  if (!P || !params || !slot || max_steps < 1) return HOSC_EINVAL;
  *slot = -1;
  const size_t need = hosc_workspace_bytes(params);
  if (need == 0) return HOSC_EINVAL;
  if (need > P->budget) return HOSC_EINVAL;            // can never fit
  if (params->inner_max != 0) return HOSC_EINVAL;      // members run captured steps only
  if (P->mode == HOSC_POOL_PERSISTENT &&
      (params->precision != HOSC_MIXED || params->solver != 0 || params->use_history != 0))
    return HOSC_EINVAL;                                 // what the round kernel runs
  if (P->used + need > P->budget) return HOSC_ENOMEM;  // fits once others retire
  PCU(cudaSetDevice(P->device));
  hosc_params p = *params;
  p.cuda_stream = nullptr;   // each member on its own stream
  void* ctx = nullptr;
  hosc_status st = hosc_create(&p, &ctx);
  if (st) return st;
  int s = -1;
  for (int q = 0; q < (int)P->m.size(); ++q)
    if (P->m[q].state == kFree) {
      s = q;
      break;
    }
  if (s < 0) {
    P->m.emplace_back();
    s = (int)P->m.size() - 1;
  }
  Member& q = P->m[s];
  if (!q.join && cudaEventCreateWithFlags(&q.join, cudaEventDisableTiming) != cudaSuccess) {
    hosc_destroy(ctx);
    return HOSC_ECUDA;
  }
  q.ctx = ctx;
  q.state = kActive;
  q.N = p.N;
  q.bytes = ctx_workspace(ctx);
  q.max_steps = max_steps;
  q.status = HOSC_OK;
  memset(&q.info, 0, sizeof(q.info));
  memset(&q.diag, 0, sizeof(q.diag));
  q.signature = -1;
  P->used += q.bytes;
  P->dirty = true;
  if (p.precision == HOSC_MIXED) {
    auto it = P->tiles.find(p.N);
    if (it != P->tiles.end()) apply_shape(ctx, it->second);
  }
  *slot = s;
  return HOSC_OK;
}

hosc_status hosc_pool_run(void* pool, int rounds, int* done_slots, int cap, int* ndone) {
  Pool* P = (Pool*)pool;
  if (!P || rounds < 1 || cap < 0 || (cap > 0 && !done_slots)) return HOSC_EINVAL;
  int nd = 0;
  PCU(cudaSetDevice(P->device));
  for (int r = 0; r < rounds && nd == 0; ++r) {
    std::vector<int> act;
    for (int q = 0; q < (int)P->m.size(); ++q)
      if (P->m[q].state == kActive) act.push_back(q);
    if (act.empty()) break;
    std::vector<hosc_status> st(act.size(), HOSC_OK);
    if (P->mode == HOSC_POOL_GRAPH) {
      if (needs_capture(P)) {
        hosc_status cs = capture_round(P);
        if (cs) return cs;
      }
      for (int q : act) ctx_begin_round(P->m[q].ctx, P->G);
      PCU(cudaGraphLaunch(P->exec, P->stream));
      PCU(cudaStreamSynchronize(P->stream));
    } else if (P->mode == HOSC_POOL_PERSISTENT) {
      std::vector<RoundMember> rm(act.size());
      for (size_t a = 0; a < act.size(); ++a) {
        void* ctx = P->m[act[a]].ctx;
        if (!ctx_persistent_ok(ctx)) return HOSC_ESTATE;
        ctx_begin_round(ctx, P->G);
        ctx_round_member(ctx, &rm[a]);
      }
      PCU(cudaDeviceSynchronize());   // the members' own streams are idle
      hosc_status rs = launch_flow(P->rs, rm, P->G, P->stream, detail_buffer(), 256);
      if (rs) return rs;
      for (size_t a = 0; a < act.size(); ++a) {
        hosc_status e = ctx_readback_round(P->m[act[a]].ctx, P->stream, P->G);
        if (e) return e;
      }
      PCU(cudaStreamSynchronize(P->stream));
    } else {
      for (size_t a = 0; a < act.size(); ++a) st[a] = ctx_enqueue_round(P->m[act[a]].ctx, P->G);
    }
    for (size_t a = 0; a < act.size(); ++a) {
      hosc_info ri;
      memset(&ri, 0, sizeof(ri));
      bool steady = false;
      hosc_status s = st[a];
      if (!s)
        s = ctx_collect_round(P->m[act[a]].ctx, P->mode == HOSC_POOL_STREAMS, &ri, &steady);
      if (s == HOSC_ECUDA) return s;   // the device is in trouble: stop the pool
      hosc_status e = settle(P, act[a], s, steady, ri, done_slots, cap, &nd);
      if (e) return e;
    }
    P->rounds += 1;
  }
  if (ndone) *ndone = nd;
  return HOSC_OK;
}

hosc_status hosc_pool_result(void* pool, int slot, hosc_status* status, hosc_info* info,
                             hosc_diag* diag, void** ctx) {
  Pool* P = (Pool*)pool;
  if (!P || slot < 0 || slot >= (int)P->m.size() || P->m[slot].state == kFree) return HOSC_EINVAL;
  const Member& q = P->m[slot];
  if (status) *status = q.state == kDone ? q.status : HOSC_ESTATE;
  if (info) *info = q.info;
  if (diag) *diag = q.diag;
  if (ctx) *ctx = q.ctx;
  return HOSC_OK;
}

hosc_status hosc_pool_retire(void* pool, int slot) {
  Pool* P = (Pool*)pool;
  if (!P || slot < 0 || slot >= (int)P->m.size() || P->m[slot].state == kFree) return HOSC_EINVAL;
  PCU(cudaSetDevice(P->device));
  Member& q = P->m[slot];
  if (P->exec) {   // the pool graph may still name this member: wait for it, then drop it
    PCU(cudaStreamSynchronize(P->stream));
    drop_exec(P);
  }
  hosc_destroy(q.ctx);
  q.ctx = nullptr;
  P->used -= q.bytes;
  q.bytes = 0;
  q.state = kFree;
  P->dirty = true;
  return HOSC_OK;
}

hosc_status hosc_pool_stats(void* pool, hosc_pool_info* out) {
  Pool* P = (Pool*)pool;
  if (!P || !out) return HOSC_EINVAL;
  memset(out, 0, sizeof(*out));
  for (const Member& q : P->m) {
    if (q.state == kActive) out->active += 1;
    if (q.state == kDone) out->completed += 1;
  }
  out->bytes_used = P->used;
  out->budget = P->budget;
  out->rounds = P->rounds;
  out->captures = P->captures;
  out->capture_ms = P->capture_ms;
  out->tuned_sizes = (int)P->tiles.size();
  return HOSC_OK;
}

}  // extern "C"
