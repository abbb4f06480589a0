// Internal declarations shared by the translation units of libhosc.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "hosc.h"

namespace hosc {

constexpr int kThreads = 256;     // threads per block of the grid-stride stencil kernels
constexpr int kRedSlots = 8;      // doubles of partial sums written per block

// Scalars that kernels take by value.
struct DevParams {
  int N;
  int newtonian;     // n == 1: eta == 1 exactly
  int have_prev;     // level n-1 history present (else delta_t^- = 0)
  int max_lin_iter;
  int sweep_fp32;    // S1-S3 arithmetic (and eta, L, E* storage) in float
  int krylov_fp32;   // right-hand sides, operator weights and Krylov vectors in float,
                     // interleaved (one float4 per node for the four systems)
  int kblock;        // interleaved Krylov kernels: threads per block (multiple of 32, 64..384)
  int kz;            // interleaved Krylov kernels: planes marched by one thread (1..N-2)
  int narrow;        // interleaved Krylov kernels compiled for 64 registers (kblock <= 256);
                     // otherwise for 80 (three-kernel form, kblock <= 384) or 128 (merged
                     // form, kblock <= 256)
  int merged;        // interleaved solve: two kernels per BiCGSTAB iteration (the x, r update
                     // folded into the next p, v kernel) instead of three
  int sx, sy, skz;   // staged stencil kernels (p/v and s/t): tile of sx * sy interior columns,
                     // skz planes per block; sx == 0 selects the register kernels instead
  int tty, ttx, tkz; // bulk-copy (TMA) stencil kernels (p/v and s/t): tile of ttx * tty interior
                     // columns, tkz planes per block; tty == 0: not used
  int tstages;       // their ring of shared-memory stages (3, 4, 6 or 8)
  int tkernels;      // which of them run: 1 p/v, 2 s/t, 3 both
  int xr_flat;       // x/r as one flat grid-stride stream (k8_xr) instead of the column march
  double h, h2;      // grid spacing along x and its square
  double Ly, Lz;     // box 1 x Ly x Lz: lengths along y and z (1 for the cube)
  // Spacing constants of the directions d = x, y, z (spacings h, k, l = h, Ly h, Lz h), in double
  // and in float (the float sweeps read them as operands): 1/(2 h_d), 1/h_d^2, h_d^2/12, 1/h_d;
  // the edge-group factors (h^2+k^2)/12, (k^2+l^2)/12, (l^2+h^2)/12; the weights of the
  // first-derivative terms of p1, q1, r1: 2k^2/(h^2+k^2), 2h^2/(h^2+k^2), 2l^2/(k^2+l^2),
  // 2k^2/(k^2+l^2), 2h^2/(l^2+h^2), 2l^2/(l^2+h^2) (all 1 when h = k = l)
  double inv2[3], isq[3], sq12[3], ih[3], grp[3], pw[6];
  float inv2f[3], isqf[3], sq12f[3], ihf[3], grpf[3], pwf[6];
  float csf[3];      // -dt/(2 h_d^2): the dt part of the symmetric weights of the compact operators
  double s3;         // (1/h^2 + 1/k^2 + 1/l^2)/3: threshold of the pseudo-time mass (1/h^2 when
                     // h = k = l)
  float s3f;
  double eta_exp;    // (n - 1)/2, the exponent of the regularised viscosity
  // float copies of the scalars the float sweeps use (converted once on the host)
  float dtf, Prf, Raf, theta_reff, I2_epsf, eta_expf, a_limitf, a_boostf;
  double iPr;          // 1/Pr, and its float copy
  float iPrf;
  double Ra, Pr, n, dt, lambda, theta_ref, I2_eps, phi, tol_div, tol_lin, a_limit, a_boost;
  int precond;         // Jacobi row scaling of the level-(n+1) systems
  int solver;          // 0: BiCGSTAB; 1: BiCGSTAB(2) (planar FP64 solve)
  int inner_pass;      // an inner pressure pass: momentum only (theta kept, its system skipped)
  int lambda_mode;     // 0: p -= lambda div V; 1: p -= min(lambda eta, lambda_cap) div V
  double lambda_cap;   // 0.9 h_min^2 / dt
  double steady_res;   // a step with max|chi^{n+1} - chi^n| below this (tol_steady * dt) and
  double div_steady;   // max|div V| below this (div_steady, else tol_div) is steady
};

constexpr int kRing = 256;   // step records kept on the device between host reads

// BiCGSTAB scalars of one system, resident in device memory.
struct KrylovScalars {
  double rho, alpha, omega, beta, r0norm, rnorm;
  double g1, g2;     // BiCGSTAB(2): minimal-residual coefficients gamma_1, gamma_2 of the cycle
  int done, iters, status, pad;
};

// What one step reports, resident in device memory (one small D2H copy per host call).
struct StepRecord {
  double res;        // max |chi^{n+1} - chi^n|
  double div_max;    // max |div V^{n+1}|
  double lin_res;    // max over systems of ||r|| / ||r_0||
  int iters[4];
  int lin_status[4];
  int status;
  int pad;
  double res_theta;  // max |theta^{n+1} - theta^n| (walls included), kept for inner passes
};

// Device arrays of one context. All N^3 doubles unless noted.
struct Fields {
  double* u[2];      // velocity, double-buffered: [cur] level n, [1-cur] level n+1 / n-1
  double* v[2];
  double* w[2];
  double* th;        // temperature
  double* p;         // pressure
  double* eta;       // apparent viscosity, level n
  double* L[2];      // 1/(Pr eta): [cur] level n, [1-cur] level n-1
  double* Eu[2];     // momentum sources E*, [cur] level n, [1-cur] level n-1
  double* Ev[2];
  double* Ew[2];
  double* Am[7];     // momentum level-(n+1) operator weights: c, x+, x-, y+, y-, z+, z-
  double* Ae[7];     // energy level-(n+1) operator weights
  double* rhs[4];    // dt (R - B chi^n) of u, v, w, theta; BiCGSTAB's fixed shadow residual
  double* x[4];      // BiCGSTAB iterate: the increment chi^{n+1} - chi^n
  double* r[4];      // residual
  double* pk[2][4];  // search direction, ping-pong
  double* vk[2][4];  // A p, ping-pong
  double* t[4];      // A s
  // BiCGSTAB(2) (solver = 1) only: u_0, r_2, u_2 of each system (null otherwise). The cycle
  // keeps r_0 in r / t (ping-pong by cycle), r_1 in pk, u_1 in vk.
  double* u0[4];
  double* r2[4];
  double* u2[4];
  double* div;       // div V^{n+1}
  double* red;       // reduction partials [blocks][kRedSlots]
  unsigned int* counter;   // last-block ticket (reset by the last block)
  KrylovScalars* ks;       // [4]
  StepRecord* rec;         // [1]
  double* diag_scal;       // diagnostics scalars
  double* nu_hot;          // [N*N] Nu_local at x = 0, index j + N*k
  double* nu_cold;         // [N*N]
  double* nu_avg;          // [N]
  double* eloc;            // [3 N^3] E_HT, E_FF, E_local (diagnostics)
  double* alg_bytes;       // [HOSC_K_COUNT] algorithmic bytes moved by each kernel class
  // device-side control of a sequence of steps enqueued without host synchronisation
  int* halt;              // 0: run; 1: a step failed; 2: steady (when *steady_stop); later
                          // kernels of the sequence return at once
  int* steady_stop;       // stop the sequence at the first steady step
  StepRecord* ring;       // [kRing] records of the steps of the sequence
  unsigned int* ring_pos; // records appended so far
  // Mixed precision solve, interleaved over the four systems (u, v, w, theta components of one
  // float4 per node). These alias the planar Krylov arrays above, which only the FP64 solve uses.
  // The two level-(n+1) operators in compact form (not row-scaled): along direction d the
  // weights of the +d and -d neighbours are S_d - B_d and S_d + B_d, with the symmetric part
  // S_d = -dt/(2 h_d^2) + L/12 for momentum (a function of L alone) and -dt/(2 h_d^2) + 1/12 for
  // energy; D is the diagonal weight.
  float4* kwm;       // momentum (B_x, B_y, B_z, D)
  float4* kwe;       // energy (B_x, B_y, B_z, D)
  float* kL;         // momentum L = 1/(Pr eta)
  float4* kr0;       // right-hand sides dt (R - B chi^n) = r_0, the shadow residual
  float4* kx;        // iterate (the increments)
  float4* kr;        // residual (the merged iteration ping-pongs it with kr1)
  float4* kr1;
  float4* kt;        // A s
  float4* kp[2];     // search direction, ping-pong
  float4* kv[2];     // A p, ping-pong
  // float copies of the state for the FP32 sweeps of mixed precision (rounded once per step)
  float* us[2];
  float* vs[2];
  float* ws[2];
  float* ths;
  float* ps;
  // host address of the tensor maps of the bulk-copy stencil kernels (kTmaMaps CUtensorMap
  // objects encoded for the context's arrays and tile shape; the launches pass them to the
  // kernels as parameters)
  const void* tmaps_host;
};

// Bytes of a context's device workspace (the BiCGSTAB(2) vectors included when bicgstab2);
// fills f when base != 0.
size_t workspace_layout(int N, int bicgstab2, Fields* f, char* base);
int red_blocks(long count);
// Rows of the per-block partials buffer of an N^3 context: enough for any launch shape the
// validation accepts (at least 32 threads per block, one plane per thread).
inline long red_rows(long n3) { return n3 / 16 + 1024; }
// Blocks of one interleaved Krylov launch (the partials buffer holds red_rows(N^3) rows).
long krylov4_blocks(const DevParams& P);
// Threads per block and planes per thread of the interleaved Krylov kernels when none are set:
// 128 threads (wide three-kernel form) and the z-segment with the least wave cost below.
void default_tiles(int N, int* kblock, int* kz);
// Waves of resident blocks a launch shape needs on this GPU times the planes each block streams
// (kz + 2): a model of the launch's duration when it is latency-bound.
double krylov4_wave_cost(int N, int kblock, int kz, int narrow, int merged, int sms);
// The same model for the staged stencil kernels with tile sx * sy and skz planes per block
// (occupancy from their shared memory and registers); infinite for a shape that cannot launch.
double staged_wave_cost(int N, int sx, int sy, int skz, int sms);
// Dynamic shared memory of a staged launch (bytes), for tile sx * sy.
size_t staged_smem_bytes(int sx, int sy, bool pv);

// Bulk-copy (TMA) stencil kernels (hosc_tma.cu). The interior columns of a plane are cut into
// tiles of ttx * tty (ttx from N: whole interior rows up to 126 columns, else the least even
// split), a block streams the tile through tkz planes.
constexpr int kTmaMaps = 8;        // kr, kr0, kp[0], kp[1], kv[0], kv[1], kwm, kwe
constexpr int kTmaMapBytes = 128;  // sizeof(CUtensorMap)
int tma_tile_x(int N);
// False when the shape does not launch (shared memory, threads, block count).
bool tma_tiles_valid(int N, int tty, int tkz, int stages);
// Encode the tensor maps of P's tile shape for F's arrays into host (kTmaMaps * 128 bytes,
// 64-byte aligned); false when the driver cannot encode them.
bool tma_prepare(const DevParams& P, const Fields& F, void* host);
double tma_wave_cost(int N, int tty, int tkz, int stages, int sms);
void launch_tma_pv(const DevParams& P, const Fields& F, int pp, cudaStream_t s);
void launch_tma_st(const DevParams& P, const Fields& F, int pp, cudaStream_t s);
long tma_blocks(const DevParams& P);
// Blocks of the flat x/r kernel (one wave of resident blocks).
int xr_flat_blocks();
int device_sms();

// S1: eta and L at every node.
void launch_viscosity(const DevParams& P, const Fields& F, int cur, cudaStream_t s);
// S2: E* of the momentum equations at every node.
void launch_sources(const DevParams& P, const Fields& F, int cur, cudaStream_t s);
// S3/S4: right-hand sides dt (R - B chi^n) and the level-(n+1) weights at interior nodes.
void launch_rhs(const DevParams& P, const Fields& F, int cur, cudaStream_t s);
// S5: BiCGSTAB pieces.
void launch_bicg_init(const DevParams& P, const Fields& F, cudaStream_t s);
void launch_bicg_pv(const DevParams& P, const Fields& F, int pp, cudaStream_t s);
void launch_bicg_st(const DevParams& P, const Fields& F, int pp, cudaStream_t s);
void launch_bicg_xr(const DevParams& P, const Fields& F, int pp, cudaStream_t s);
// BiCGSTAB(2), planar FP64 solve: the five kernels of one cycle, r_0 ping-pong parity cp
// (launch_bicg_init starts the solve for either solver).
void launch_b2(int kernel, const DevParams& P, const Fields& F, int cp, cudaStream_t s);
// Mark all four systems as iterating (for timing the Krylov kernels in isolation).
void launch_krylov_activate(const Fields& F, cudaStream_t s);
// Body of the BiCGSTAB loop of a captured step: end of the loop when every system is done.
void launch_loop_cond(const Fields& F, unsigned long long handle, cudaStream_t s);
// S6-S8: increments, theta walls, div V, pressure correction and walls, step record.
void launch_update(const DevParams& P, const Fields& F, int cur, cudaStream_t s);
// The same without the step record (an inner pressure pass follows), and the record alone.
void launch_update_fields(const DevParams& P, const Fields& F, int cur, cudaStream_t s);
void launch_finish(const DevParams& P, const Fields& F, cudaStream_t s);
// Re-arm the device control of a sequence of steps: run (halt = 0), no records yet, and stop at
// the first steady step when stop_steady.
void launch_arm(const Fields& F, int stop_steady, cudaStream_t s);
// Mixed precision: round u, v, w (level cur, and level 1-cur when both), theta and p to float.
void launch_shadow(const DevParams& P, const Fields& F, int cur, int both, cudaStream_t s);
// Diagnostics.
void launch_diagnostics(const DevParams& P, const Fields& F, int cur, int want_fields,
                        cudaStream_t s);

// One member of a persistent round (hosc_round.cu): its parameters (launch shape of the Krylov
// tiles set for the round kernel), arrays, level of the round's first step, and the number of
// 256-thread items of each phase.
struct RoundMember {
  DevParams P;
  Fields F;
  int cur;
  int nodes;           // N^3 nodes
  int interior;        // (N-2)^3 interior nodes
  int theta_walls;     // adiabatic wall nodes with x interior
  int pressure_walls;  // boundary nodes
  int kx, ky;          // Krylov tiles: column chunks x plane segments
  int init;            // blocks of the Krylov initialisation (a grid-stride loop)
};
struct RoundState;
RoundState* round_state_create();
void round_state_destroy(RoundState* S);
// Items and Krylov tile shape of a member (sets P.kblock, P.kz for the round kernel).
void round_member_shape(RoundMember* M);
// One persistent round of G steps of every member on `stream` (one cooperative launch), waited
// for: each member advances through its own phases, whose tiles any block takes from a shared
// queue. HOSC_ECUDA with detail on a CUDA error or when a queue wait gave up; HOSC_ENOMEM when
// one phase of all members has more tiles than the queue holds.
hosc_status launch_flow(RoundState* S, const std::vector<RoundMember>& members, int G,
                        cudaStream_t stream, char* detail, size_t detail_len);

// Rounds of captured steps of one context, driven by a pool (hosc_pool.cu); defined with the
// context in hosc_api.cu. ctx is a context made by hosc_create.
char* detail_buffer();                       // text returned by hosc_last_error_detail
size_t ctx_workspace(void* ctx);             // device bytes the context holds
int ctx_N(void* ctx);
cudaStream_t ctx_branch_stream(void* ctx);   // stream on which ctx_append_round captures
long ctx_signature(void* ctx);               // changes when a captured round no longer applies
void ctx_begin_round(void* ctx, long n);
hosc_status ctx_enqueue_round(void* ctx, int n);
hosc_status ctx_append_round(void* ctx, int n);
hosc_status ctx_collect_round(void* ctx, bool wait, hosc_info* info, bool* steady);
// Persistent rounds: whether the context can run in one (mixed precision, BiCGSTAB, no history,
// no inner passes, captured steps usable), its round member (after ctx_begin_round), and the
// asynchronous read-back of its records on `s` once the round kernel has run.
bool ctx_persistent_ok(void* ctx);
void ctx_round_member(void* ctx, RoundMember* out);
hosc_status ctx_readback_round(void* ctx, cudaStream_t s, int n);

}  // namespace hosc
