// Internal declarations shared by the translation units of libhosc.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
  int krylov_fp32;   // right-hand sides, operator weights and Krylov vectors in float
  double h, h2;      // grid spacing (h = k = l) and its square
  double Ra, Pr, n, dt, lambda, theta_ref, I2_eps, phi, tol_div, tol_lin, a_limit, a_boost;
  double steady_res;   // a step with max|chi^{n+1} - chi^n| below this (and div below tol_div)
                       // is steady (tol_steady * dt)
};

constexpr int kRing = 256;   // step records kept on the device between host reads

// BiCGSTAB scalars of one system, resident in device memory.
struct KrylovScalars {
  double rho, alpha, omega, beta, r0norm, rnorm;
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
  // float copies of the state for the FP32 sweeps of mixed precision (rounded once per step)
  float* us[2];
  float* vs[2];
  float* ws[2];
  float* ths;
  float* ps;
};

size_t workspace_layout(int N, Fields* f, char* base);   // returns bytes; fills f when base != 0
int red_blocks(long count);

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
// Body of the BiCGSTAB loop of a captured step: end of the loop when every system is done.
void launch_loop_cond(const Fields& F, unsigned long long handle, cudaStream_t s);
// S6-S8: increments, theta walls, div V, pressure correction and walls, step record.
void launch_update(const DevParams& P, const Fields& F, int cur, cudaStream_t s);
// Mixed precision: round u, v, w (level cur, and level 1-cur when both), theta and p to float.
void launch_shadow(const DevParams& P, const Fields& F, int cur, int both, cudaStream_t s);
// Diagnostics.
void launch_diagnostics(const DevParams& P, const Fields& F, int cur, int want_fields,
                        cudaStream_t s);

}  // namespace hosc
