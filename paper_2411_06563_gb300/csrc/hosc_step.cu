// Launchers of the step kernels other than the Krylov solver (Punia & Ray, arXiv:2411.06563,
// Sec. 2.2): viscosity (S1), momentum sources (S2), compact right-hand sides and level-(n+1)
// operator weights (S3/S4), increments, wall conditions, divergence and the modified
// artificial-compressibility pressure correction (S6-S8). The device code is in
// hosc_step_dev.cuh; one block of kThreads threads per 256 nodes.

#include <math.h>

#include "hosc_step_dev.cuh"

namespace hosc {

void launch_arm(const Fields& F, int stop_steady, cudaStream_t s) {
  k_arm<<<1, 32, 0, s>>>(F.halt, F.ring_pos, F.steady_stop, stop_steady);
}

int red_blocks(long count) { return (int)((count + kThreads - 1) / kThreads); }


void launch_shadow(const DevParams& P, const Fields& F, int cur, int both, cudaStream_t s) {
  const int n3 = P.N * P.N * P.N;
  k_shadow<<<red_blocks(n3), kThreads, 0, s>>>(n3, F.u[cur], F.v[cur], F.w[cur], F.th, F.p,
                                               F.us[cur], F.vs[cur], F.ws[cur], F.ths, F.ps, F.halt);
  if (both) {
    const int o = 1 - cur;
    k_shadow<<<red_blocks(n3), kThreads, 0, s>>>(n3, F.u[o], F.v[o], F.w[o], nullptr, nullptr,
                                                 F.us[o], F.vs[o], F.ws[o], nullptr, nullptr,
                                                 F.halt);
  }
}

void launch_viscosity(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long n3 = (long)P.N * P.N * P.N;
  if (P.sweep_fp32)
    k_viscosity<float><<<red_blocks(n3), kThreads, 0, s>>>(
        P, F.us[cur], F.vs[cur], F.ws[cur], reinterpret_cast<float*>(F.eta),
        reinterpret_cast<float*>(F.L[cur]), F.halt);
  else
    k_viscosity<double><<<red_blocks(n3), kThreads, 0, s>>>(P, F.u[cur], F.v[cur], F.w[cur],
                                                            F.eta, F.L[cur], F.halt);
}

void launch_sources(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long n3 = (long)P.N * P.N * P.N;
  if (P.sweep_fp32)
    k_sources<float><<<red_blocks(n3), kThreads, 0, s>>>(
        P, F.us[cur], F.vs[cur], F.ws[cur], F.ths, F.ps, reinterpret_cast<const float*>(F.eta),
        reinterpret_cast<float*>(F.Eu[cur]), reinterpret_cast<float*>(F.Ev[cur]),
        reinterpret_cast<float*>(F.Ew[cur]), F.halt);
  else
    k_sources<double><<<red_blocks(n3), kThreads, 0, s>>>(P, F.u[cur], F.v[cur], F.w[cur], F.th,
                                                          F.p, F.eta, F.Eu[cur], F.Ev[cur],
                                                          F.Ew[cur], F.halt);
}

template <class Tc, class Ts>
static void rhs_t(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long ni = P.N - 2;
  const int o = 1 - cur;
  auto T = [](double* p) { return reinterpret_cast<const Tc*>(p); };
  // the state: float copies for FP32 sweeps, the double arrays otherwise
  const Tc *u, *v, *w, *th, *up, *vp, *wp;
  if (sizeof(Tc) == sizeof(float)) {
    u = (const Tc*)F.us[cur]; v = (const Tc*)F.vs[cur]; w = (const Tc*)F.ws[cur];
    th = (const Tc*)F.ths;
    up = (const Tc*)F.us[o]; vp = (const Tc*)F.vs[o]; wp = (const Tc*)F.ws[o];
  } else {
    u = (const Tc*)F.u[cur]; v = (const Tc*)F.v[cur]; w = (const Tc*)F.w[cur];
    th = (const Tc*)F.th;
    up = (const Tc*)F.u[o]; vp = (const Tc*)F.v[o]; wp = (const Tc*)F.w[o];
  }
  k_rhs<Tc, Ts><<<red_blocks(ni * ni * ni), kThreads, 0, s>>>(
      P, u, v, w, th, T(F.L[cur]), T(F.Eu[cur]), T(F.Ev[cur]), T(F.Ew[cur]), T(F.L[o]), up, vp,
      wp, T(F.Eu[o]), T(F.Ev[o]), T(F.Ew[o]), F);
}

void launch_rhs(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  if (P.sweep_fp32)
    rhs_t<float, float>(P, F, cur, s);
  else if (P.krylov_fp32)
    rhs_t<double, float>(P, F, cur, s);
  else
    rhs_t<double, double>(P, F, cur, s);
}

void launch_update(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  launch_update_fields(P, F, cur, s);
  launch_finish(P, F, s);
}

void launch_finish(const DevParams& P, const Fields& F, cudaStream_t s) {
  k_finish_record<<<1, 32, 0, s>>>(P, F);
}

void launch_update_fields(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long N = P.N, n3 = N * N * N, ni = N - 2;
  const int b_all = red_blocks(n3);
  if (P.krylov_fp32)
    k_apply_increment<float><<<b_all, kThreads, 0, s>>>(P, F, cur, b_all);
  else
    k_apply_increment<double><<<b_all, kThreads, 0, s>>>(P, F, cur, b_all);
  const int b_walls = red_blocks(2 * ni * N + 2 * ni * ni);
  k_theta_walls<<<b_walls, kThreads, 0, s>>>(P, F, b_walls);
  const int b_int = red_blocks(ni * ni * ni);
  k_divergence<<<b_int, kThreads, 0, s>>>(P, F, 1 - cur, b_int);
  k_pressure_correct<<<b_int, kThreads, 0, s>>>(P, F);
  k_pressure_walls<<<red_blocks(n3 - ni * ni * ni), kThreads, 0, s>>>(P, F);
}

}  // namespace hosc
