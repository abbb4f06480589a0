// hosc_bicgstab_noalloc: the BiCGSTAB solve of the four level-(n+1) systems of one step without
// any device allocation. The Krylov vectors, reduction partials and solver scalars live in one
// file-scope device array of fixed size (HOSC_NOALLOC_MAX_N nodes per side), shared by every call
// in the process; inputs and outputs are the caller's device arrays. The kernels are the ones of
// the context path (hosc_krylov.cu), so the result equals the context's solve. The host checks
// convergence every 4 to 16 iterations: it copies the four systems' solver scalars to the host and
// synchronises the stream, so a call returns only once its solve has finished.

#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "hosc.h"
#include "hosc_internal.h"

using namespace hosc;

namespace {

constexpr int kMaxN = HOSC_NOALLOC_MAX_N;
constexpr size_t kMaxNodes = (size_t)kMaxN * kMaxN * kMaxN;
constexpr size_t kVecBytes = kMaxNodes * sizeof(double);
constexpr size_t kAlignB = 256;
// 6 vectors (r, p x2, v x2, t) for each of the 4 systems, then the small control block.
constexpr size_t kVectorsBytes = 24 * ((kVecBytes + kAlignB - 1) / kAlignB * kAlignB);
constexpr size_t kMaxBlocks = (kMaxNodes + kThreads - 1) / kThreads;
constexpr size_t kControlBytes = 64 * 1024 + kMaxBlocks * kRedSlots * sizeof(double);
constexpr size_t kScratchBytes = kVectorsBytes + kControlBytes;
// Offsets of the control block: solver scalars at 0, ticket counter at 512, halt flag at 768,
// per-kernel byte counters at 1024, reduction partials from 4096 on.
constexpr size_t kOffCounter = 512, kOffHalt = 768, kOffBytes = 1024, kOffRed = 4096;
static_assert(4 * sizeof(KrylovScalars) <= kOffCounter, "solver scalars overlap the counter");
static_assert(kOffCounter + sizeof(unsigned int) <= kOffHalt, "counter overlaps the halt flag");
static_assert(kOffHalt + sizeof(int) <= kOffBytes, "halt flag overlaps the byte counters");
static_assert(kOffBytes + HOSC_K_COUNT * sizeof(double) <= kOffRed,
              "byte counters overlap the reduction partials");
static_assert(kOffRed + kMaxBlocks * kRedSlots * sizeof(double) <= kControlBytes,
              "reduction partials exceed the control block");

// The scratch. In host code this name is only a stand-in for the symbol: its device address comes
// from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_addr[64] = {};   // device address of g_scratch, per device ordinal

hosc_status scratch_address(int device, char** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (device < 0 || device >= 64) return HOSC_EINVAL;
  if (!g_addr[device]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) return HOSC_ECUDA;
    g_addr[device] = ptr;
  }
  *out = (char*)g_addr[device];
  return HOSC_OK;
}

}  // namespace

extern "C" hosc_status hosc_bicgstab_noalloc(int N, const double* const* weights,
                                             const double* const* rhs, double* const* x,
                                             double tol, int max_iter, int* iters_out,
                                             void* stream) {
  if (N < 5 || N > kMaxN) return HOSC_EINVAL;
  if (!weights || !rhs || !x || !(tol > 0.0) || max_iter < 1) return HOSC_EINVAL;
  for (int q = 0; q < 14; ++q)
    if (!weights[q]) return HOSC_EINVAL;
  for (int s = 0; s < 4; ++s)
    if (!rhs[s] || !x[s]) return HOSC_EINVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return HOSC_ECUDA;
  char* base = nullptr;
  hosc_status st = scratch_address(device, &base);
  if (st) return st;
  cudaStream_t sm = (cudaStream_t)stream;

  // Carve the scratch: vectors sized for this N, then the control block.
  const size_t n3 = (size_t)N * N * N;
  const size_t vb = (n3 * sizeof(double) + kAlignB - 1) / kAlignB * kAlignB;
  Fields F;
  memset(&F, 0, sizeof(F));
  char* p = base;
  for (int s = 0; s < 4; ++s) {
    F.r[s] = (double*)p; p += vb;
    F.t[s] = (double*)p; p += vb;
    for (int b = 0; b < 2; ++b) {
      F.pk[b][s] = (double*)p; p += vb;
      F.vk[b][s] = (double*)p; p += vb;
    }
  }
  const size_t vec_used = (size_t)(p - base);
  char* ctl = base + kVectorsBytes;
  F.ks = (KrylovScalars*)ctl;                      // 4 x sizeof(KrylovScalars) = 320 bytes
  F.counter = (unsigned int*)(ctl + kOffCounter);
  F.halt = (int*)(ctl + kOffHalt);
  F.alg_bytes = (double*)(ctl + kOffBytes);
  F.red = (double*)(ctl + kOffRed);
  for (int q = 0; q < 7; ++q) {
    F.Am[q] = const_cast<double*>(weights[q]);
    F.Ae[q] = const_cast<double*>(weights[7 + q]);
  }
  for (int s = 0; s < 4; ++s) {
    F.rhs[s] = const_cast<double*>(rhs[s]);
    F.x[s] = x[s];
  }
  // Every call shares the scratch and finds the previous call's contents: the vectors must read
  // zero on the walls and the ticket counter and halt flag must start at zero.
  if (cudaMemsetAsync(base, 0, vec_used, sm) != cudaSuccess) return HOSC_ECUDA;
  if (cudaMemsetAsync(ctl, 0, kOffRed, sm) != cudaSuccess) return HOSC_ECUDA;

  DevParams P;
  memset(&P, 0, sizeof(P));
  P.N = N;
  P.max_lin_iter = max_iter;
  P.tol_lin = tol;
  P.h = 1.0 / (N - 1);
  P.h2 = P.h * P.h;

  KrylovScalars ks[4];
  launch_bicg_init(P, F, sm);
  int pp = 0, it = 0, check = 4;
  while (it < max_iter) {
    const int chunk = (max_iter - it < check) ? max_iter - it : check;
    for (int q = 0; q < chunk; ++q) {
      launch_bicg_pv(P, F, pp, sm);
      launch_bicg_st(P, F, pp, sm);
      launch_bicg_xr(P, F, pp, sm);
      pp ^= 1;
    }
    it += chunk;
    if (cudaGetLastError() != cudaSuccess) return HOSC_ECUDA;
    if (cudaMemcpyAsync(ks, F.ks, sizeof(ks), cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        cudaStreamSynchronize(sm) != cudaSuccess)
      return HOSC_ECUDA;
    if (ks[0].done && ks[1].done && ks[2].done && ks[3].done) break;
    if (check < 16) check *= 2;
  }
  st = HOSC_OK;
  for (int s = 0; s < 4; ++s) {
    if (iters_out) iters_out[s] = ks[s].iters;
    if (ks[s].status != 0 || !ks[s].done) st = HOSC_ENOCONV;
  }
  return st;
}
