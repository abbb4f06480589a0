// Kernels of one HOSC pseudo-time step except the Krylov solver (Punia & Ray, arXiv:2411.06563,
// Sec. 2.2): viscosity (S1), momentum sources (S2), compact right-hand sides and level-(n+1)
// operator weights (S3/S4), increments, wall conditions, divergence and the modified
// artificial-compressibility pressure correction (S6-S8).
//
// Layout: every field is N^3 doubles, x fastest (node (i,j,k) at i + N*(j + N*k)). One thread per
// node; node-linear thread indexing keeps consecutive threads on consecutive x.

#include <math.h>

#include "hosc_device.cuh"
#include "hosc_internal.h"

namespace hosc {

namespace {

__device__ __forceinline__ int inward(int a, int N) { return a == 0 ? 1 : (a == N - 1 ? N - 2 : a); }
__device__ __forceinline__ int on_wall(int a, int N) { return (a == 0) | (a == N - 1); }

// ------------------------------------------------------------------------------------ S1

// eta = (I2 + eps)^((n-1)/2) (Eqs. 7-8), eta == 1 for n == 1; L = 1/(Pr eta) (Sec. 2.2 momentum
// coefficients). On cube edges and corners, where the one-sided strain rates of two or three
// no-slip walls vanish identically, I2 is taken at the node one step inward along each of those
// wall normals.
__global__ void __launch_bounds__(kThreads) k_viscosity(DevParams P, const double* __restrict__ u,
                                                        const double* __restrict__ v,
                                                        const double* __restrict__ w,
                                                        double* __restrict__ eta,
                                                        double* __restrict__ L) {
  const int N = P.N;
  const long n3 = (long)N * N * N;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  int i = (int)(t % N), j = (int)((t / N) % N), k = (int)(t / ((long)N * N));
  double e = 1.0;
  if (!P.newtonian) {
    if (on_wall(i, N) + on_wall(j, N) + on_wall(k, N) >= 2) {
      i = inward(i, N);
      j = inward(j, N);
      k = inward(k, N);
    }
    const Grad9 g = velocity_gradients(u, v, w, i, j, k, N, 0.5 / P.h);
    e = pow(second_invariant(g) + P.I2_eps, 0.5 * (P.n - 1.0));
  }
  eta[t] = e;
  L[t] = 1.0 / (P.Pr * e);
}

// ------------------------------------------------------------------------------------ S2

// E* of the x, y, z momentum equations: the conservative momentum equations divided through by
// Pr eta so that L = 1/(Pr eta):
//   E*_x = -p_x/(Pr eta) + (2/eta)(eps_xx eta_x + eps_yx eta_y + eps_zx eta_z)
//   E*_y = -p_y/(Pr eta) + (2/eta)(eps_xy eta_x + eps_yy eta_y + eps_zy eta_z) + Ra (theta - theta_ref)/eta
//   E*_z = -p_z/(Pr eta) + (2/eta)(eps_xz eta_x + eps_yz eta_y + eps_zz eta_z)
// Gradients are central inside and one-sided at wall nodes.
__global__ void __launch_bounds__(kThreads) k_sources(DevParams P, const double* __restrict__ u,
                                                     const double* __restrict__ v,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ th,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ eta,
                                                     double* __restrict__ Eu,
                                                     double* __restrict__ Ev,
                                                     double* __restrict__ Ew) {
  const int N = P.N;
  const long n3 = (long)N * N * N;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  const int i = (int)(t % N), j = (int)((t / N) % N), k = (int)(t / ((long)N * N));
  const double inv2h = 0.5 / P.h;
  const long sy = N, sz = (long)N * N;
  const Grad9 g = velocity_gradients(u, v, w, i, j, k, N, inv2h);
  const double ex = grad_axis(eta, t, i, N, 1, inv2h);
  const double ey = grad_axis(eta, t, j, N, sy, inv2h);
  const double ez = grad_axis(eta, t, k, N, sz, inv2h);
  const double px = grad_axis(p, t, i, N, 1, inv2h);
  const double py = grad_axis(p, t, j, N, sy, inv2h);
  const double pz = grad_axis(p, t, k, N, sz, inv2h);
  const double e = eta[t];
  const double exy = 0.5 * (g.uy + g.vx), exz = 0.5 * (g.uz + g.wx), eyz = 0.5 * (g.vz + g.wy);
  const double a = 1.0 / (P.Pr * e), b = 2.0 / e;
  Eu[t] = -px * a + b * (g.ux * ex + exy * ey + exz * ez);
  Ev[t] = -py * a + b * (exy * ex + g.vy * ey + eyz * ez) + P.Ra * (th[t] - P.theta_ref) / e;
  Ew[t] = -pz * a + b * (exz * ex + eyz * ey + g.wz * ez);
}

// ------------------------------------------------------------------------------------ S3/S4

// 7-point neighbourhood order: centre, x+, x-, y+, y-, z+, z-.
struct D7 {
  double dx, dy, dz, dxx, dyy, dzz;
};

__device__ __forceinline__ D7 diffs7(const double f[7], double inv2h, double invh2) {
  D7 d;
  d.dx = (f[1] - f[2]) * inv2h;
  d.dy = (f[3] - f[4]) * inv2h;
  d.dz = (f[5] - f[6]) * inv2h;
  d.dxx = (f[1] - 2.0 * f[0] + f[2]) * invh2;
  d.dyy = (f[3] - 2.0 * f[0] + f[4]) * invh2;
  d.dzz = (f[5] - 2.0 * f[0] + f[6]) * invh2;
  return d;
}

__device__ __forceinline__ void load7(const double* __restrict__ a, long c, long sy, long sz,
                                      double f[7]) {
  f[0] = a[c];
  f[1] = a[c + 1];
  f[2] = a[c - 1];
  f[3] = a[c + sy];
  f[4] = a[c - sy];
  f[5] = a[c + sz];
  f[6] = a[c - sz];
}

// 19-point neighbourhood: 0 c, 1 x+, 2 x-, 3 y+, 4 y-, 5 z+, 6 z-,
// 7 x+y+, 8 x-y+, 9 x+y-, 10 x-y-, 11 y+z+, 12 y-z+, 13 y+z-, 14 y-z-,
// 15 z+x+, 16 z-x+, 17 z+x-, 18 z-x-.
__device__ __forceinline__ void load19(const double* __restrict__ a, long c, long sy, long sz,
                                       double f[19]) {
  load7(a, c, sy, sz, f);
  f[7] = a[c + 1 + sy];
  f[8] = a[c - 1 + sy];
  f[9] = a[c + 1 - sy];
  f[10] = a[c - 1 - sy];
  f[11] = a[c + sy + sz];
  f[12] = a[c - sy + sz];
  f[13] = a[c + sy - sz];
  f[14] = a[c - sy - sz];
  f[15] = a[c + sz + 1];
  f[16] = a[c - sz + 1];
  f[17] = a[c + sz - 1];
  f[18] = a[c - sz - 1];
}

// One edge group of Eq. (5) on a uniform grid, directions (a, b):
//   da^2 db^2 chi - Vb da^2 db chi - Va da db^2 chi - c1 da db chi
// F[pp], F[0p], F[mp], F[p0], F[00], F[m0], F[pm], F[0m], F[mm] (first index along a).
__device__ __forceinline__ double edge_group(double Fpp, double F0p, double Fmp, double Fp0,
                                             double F00, double Fm0, double Fpm, double F0m,
                                             double Fmm, double Va, double Vb, double c1,
                                             double h) {
  const double ih = 1.0 / h;
  const double ih2 = ih * ih;
  const double d22 = (Fpp + Fmp + Fpm + Fmm - 2.0 * (F0p + F0m + Fp0 + Fm0) + 4.0 * F00) * ih2 * ih2;
  const double d21 = ((Fpp - 2.0 * F0p + Fmp) - (Fpm - 2.0 * F0m + Fmm)) * (0.5 * ih2 * ih);
  const double d12 = ((Fpp - 2.0 * Fp0 + Fpm) - (Fmp - 2.0 * Fm0 + Fmm)) * (0.5 * ih2 * ih);
  const double d11 = (Fpp - Fmp - Fpm + Fmm) * (0.25 * ih2);
  return d22 - Vb * d21 - Va * d12 - c1 * d11;
}

// Coefficients of Eq. (5) shared by the systems with the same G*, H*, I* (K* = 0).
struct Eq5 {
  double G, H, I, al, be, ga, M1, M2, M3, p1, q1, r1;
};

// [1 + (dx^2 - G dx) h^2/12 + (dy^2 - H dy) k^2/12 + (dz^2 - I dz) l^2/12 + (dt/2) dt^-] f
__device__ __forceinline__ double bracket(const double f[7], double f_prev, const Eq5& c,
                                          double inv2h, double invh2, double h2_12) {
  const D7 d = diffs7(f, inv2h, invh2);
  return f[0] + h2_12 * ((d.dxx - c.G * d.dx) + (d.dyy - c.H * d.dy) + (d.dzz - c.I * d.dz)) +
         0.5 * (f[0] - f_prev);
}

__device__ __forceinline__ Eq5 eq5_coefficients(const double G7[7], const double H7[7],
                                                const double I7[7], double Gp, double Hp,
                                                double Ip, double inv2h, double invh2,
                                                double h2_12) {
  Eq5 c;
  c.G = G7[0];
  c.H = H7[0];
  c.I = I7[0];
  const D7 dG = diffs7(G7, inv2h, invh2), dH = diffs7(H7, inv2h, invh2),
           dI = diffs7(I7, inv2h, invh2);
  c.al = 1.0 + h2_12 * (c.G * c.G - 2.0 * dG.dx);
  c.be = 1.0 + h2_12 * (c.H * c.H - 2.0 * dH.dy);
  c.ga = 1.0 + h2_12 * (c.I * c.I - 2.0 * dI.dz);
  c.M1 = bracket(G7, Gp, c, inv2h, invh2, h2_12);
  c.M2 = bracket(H7, Hp, c, inv2h, invh2, h2_12);
  c.M3 = bracket(I7, Ip, c, inv2h, invh2, h2_12);
  // p1, q1, r1 with h = k = l: -G H + 2/(h^2+k^2) (k^2 dy G + h^2 dx H) = -G H + dy G + dx H
  c.p1 = -c.G * c.H + (dG.dy + dH.dx);
  c.q1 = -c.H * c.I + (dH.dz + dI.dy);
  c.r1 = -c.I * c.G + (dI.dx + dG.dz);
  return c;
}

// The level-n operator of Eq. (5) applied to chi (19 points):
//  -al dx^2 - be dy^2 - ga dz^2 + M1 dx + M2 dy + M3 dz
//  - (h^2/6) [yz group + xy group + zx group]
__device__ __forceinline__ double applyB(const Eq5& c, const double f[19], double h, double inv2h,
                                         double invh2) {
  const D7 d = diffs7(f, inv2h, invh2);
  const double gxy = edge_group(f[7], f[3], f[8], f[1], f[0], f[2], f[9], f[4], f[10], c.G, c.H,
                                c.p1, h);
  const double gyz = edge_group(f[11], f[5], f[12], f[3], f[0], f[4], f[13], f[6], f[14], c.H,
                                c.I, c.q1, h);
  const double gzx = edge_group(f[15], f[1], f[16], f[5], f[0], f[6], f[17], f[2], f[18], c.I,
                                c.G, c.r1, h);
  const double m5 = h * h / 6.0;
  return -c.al * d.dxx - c.be * d.dyy - c.ga * d.dzz + c.M1 * d.dx + c.M2 * d.dy + c.M3 * d.dz -
         m5 * (gyz + gxy + gzx);
}

// Diagonal pseudo-time mass where the cell Reynolds number is high: the level-n operator carries
// (h^2/12)|G*|^2 delta^2 explicitly, and for the grid mode alternating in all three directions the
// level-(n+1) operator is only 6 dt/h^2, so that mode grows once |G*|^2 h^2 > 24 (and the mode
// alternating in one direction once dt |G*|^2 > 4 L). Zero in resolved flows; it changes the
// pseudo-time path only, never the steady state.
__device__ __forceinline__ double pseudo_time_mass(double G, double H, double I, double L,
                                                   double dt, double invh2, double kappa) {
  const double g2 = G * G + H * H + I * I;
  const double s = fmax(0.0, fmax(dt * (g2 / 6.0 - invh2), dt * g2 / 6.0 - 2.0 * L / 3.0));
  return kappa * s;
}

// Right-hand sides of the increment form of Eq. (6),  A (chi^{n+1} - chi^n) = dt (R - B chi^n),
// for u, v, w, theta at interior nodes, and the seven level-(n+1) weights L1..L7 of the momentum
// and energy systems.
__global__ void __launch_bounds__(kThreads) k_rhs(
    DevParams P, const double* __restrict__ u, const double* __restrict__ v,
    const double* __restrict__ w, const double* __restrict__ th, const double* __restrict__ L,
    const double* __restrict__ Eu, const double* __restrict__ Ev, const double* __restrict__ Ew,
    const double* __restrict__ Lp, const double* __restrict__ up, const double* __restrict__ vp,
    const double* __restrict__ wp, const double* __restrict__ Eup,
    const double* __restrict__ Evp, const double* __restrict__ Ewp, Fields F) {
  const int N = P.N, ni = N - 2;
  const long cnt = (long)ni * ni * ni;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int i = 1 + (int)(t % ni), j = 1 + (int)((t / ni) % ni), k = 1 + (int)(t / ((long)ni * ni));
  const long sy = N, sz = (long)N * N;
  const long c = node(i, j, k, N);
  const double h = P.h, h2 = P.h2, inv2h = 0.5 / h, invh2 = 1.0 / h2, h2_12 = h2 / 12.0;
  const double dt = P.dt;

  double L7[7], u7[7], v7[7], w7[7];
  load7(L, c, sy, sz, L7);
  load7(u, c, sy, sz, u7);
  load7(v, c, sy, sz, v7);
  load7(w, c, sy, sz, w7);
  const double Lc = L7[0];
  const double Lpc = P.have_prev ? Lp[c] : Lc;
  const double upc = P.have_prev ? up[c] : u7[0];
  const double vpc = P.have_prev ? vp[c] : v7[0];
  const double wpc = P.have_prev ? wp[c] : w7[0];

  // ---------------- momentum: L = 1/(Pr eta), G* = u L, H* = v L, I* = w L, K* = 0
  {
    double G7[7], H7[7], I7[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      G7[q] = u7[q] * L7[q];
      H7[q] = v7[q] * L7[q];
      I7[q] = w7[q] * L7[q];
    }
    const Eq5 cm = eq5_coefficients(G7, H7, I7, upc * Lpc, vpc * Lpc, wpc * Lpc, inv2h, invh2, h2_12);
    const double* E[3] = {Eu, Ev, Ew};
    const double* Ep[3] = {Eup, Evp, Ewp};
    const double* X[3] = {u, v, w};
#pragma unroll 1
    for (int s = 0; s < 3; ++s) {
      double E7[7], f19[19];
      load7(E[s], c, sy, sz, E7);
      const double Epc = P.have_prev ? Ep[s][c] : E7[0];
      const double R = bracket(E7, Epc, cm, inv2h, invh2, h2_12);
      load19(X[s], c, sy, sz, f19);
      F.rhs[s][c] = dt * (R - applyB(cm, f19, h, inv2h, invh2));
    }
    // level-(n+1) weights (Eq. 6): Mx = -dt/(2L) + h^2/12, M15 = (h^2/(6L)) dx L, ...
    const D7 dL = diffs7(L7, inv2h, invh2);
    const double M = -dt / (2.0 * Lc) + h2_12;
    const double m15 = h2 / (6.0 * Lc) * dL.dx, m16 = h2 / (6.0 * Lc) * dL.dy,
                 m17 = h2 / (6.0 * Lc) * dL.dz;
    double M18 = 0.5 * (Lc - Lpc) + h2_12 * ((dL.dxx - cm.G * dL.dx) +
                                             (dL.dyy - cm.H * dL.dy) +
                                             (dL.dzz - cm.I * dL.dz));
    // keep the extrapolated mass positive where L changes fast (the steady state is unaffected)
    if (P.a_limit > 0.0) M18 = fmax(M18, -P.a_limit * Lc);
    const double a2 = M * invh2;
    const double sig_m = P.a_boost > 0.0
                             ? pseudo_time_mass(cm.G, cm.H, cm.I, Lc, dt, invh2, P.a_boost) : 0.0;
    F.Am[0][c] = Lc * (1.0 - 6.0 * a2) + M18 + sig_m;
    F.Am[1][c] = Lc * (a2 - M * cm.G * inv2h + m15 * inv2h);
    F.Am[2][c] = Lc * (a2 + M * cm.G * inv2h - m15 * inv2h);
    F.Am[3][c] = Lc * (a2 - M * cm.H * inv2h + m16 * inv2h);
    F.Am[4][c] = Lc * (a2 + M * cm.H * inv2h - m16 * inv2h);
    F.Am[5][c] = Lc * (a2 - M * cm.I * inv2h + m17 * inv2h);
    F.Am[6][c] = Lc * (a2 + M * cm.I * inv2h - m17 * inv2h);
  }
  // ---------------- energy: L = 1, G* = u, H* = v, I* = w, K* = E* = 0
  {
    const Eq5 ce = eq5_coefficients(u7, v7, w7, upc, vpc, wpc, inv2h, invh2, h2_12);
    double f19[19];
    load19(th, c, sy, sz, f19);
    F.rhs[3][c] = -dt * applyB(ce, f19, h, inv2h, invh2);
    const double M = -0.5 * dt + h2_12;
    const double a2 = M * invh2;
    const double sig_e = P.a_boost > 0.0
                             ? pseudo_time_mass(ce.G, ce.H, ce.I, 1.0, dt, invh2, P.a_boost) : 0.0;
    F.Ae[0][c] = 1.0 - 6.0 * a2 + sig_e;
    F.Ae[1][c] = a2 - M * ce.G * inv2h;
    F.Ae[2][c] = a2 + M * ce.G * inv2h;
    F.Ae[3][c] = a2 - M * ce.H * inv2h;
    F.Ae[4][c] = a2 + M * ce.H * inv2h;
    F.Ae[5][c] = a2 - M * ce.I * inv2h;
    F.Ae[6][c] = a2 + M * ce.I * inv2h;
  }
}

// ------------------------------------------------------------------------------------ S6-S8

__device__ __forceinline__ double absfin(double x) { return isfinite(x) ? fabs(x) : INFINITY; }

// chi^{n+1} = chi^n + x at interior nodes (u, v, w into the other buffer, theta in place); wall
// velocities are carried over. Max |x| over the four systems goes to the step record.
__global__ void __launch_bounds__(kThreads) k_apply_increment(DevParams P, Fields F, int cur,
                                                              int nblocks) {
  __shared__ double smem[32];
  const int N = P.N;
  const long n3 = (long)N * N * N;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double m[1] = {0.0};
  if (t < n3) {
    const int i = (int)(t % N), j = (int)((t / N) % N), k = (int)(t / ((long)N * N));
    const bool inner = i > 0 && j > 0 && k > 0 && i < N - 1 && j < N - 1 && k < N - 1;
    if (inner) {
      const double xu = F.x[0][t], xv = F.x[1][t], xw = F.x[2][t], xt = F.x[3][t];
      F.u[1 - cur][t] = F.u[cur][t] + xu;
      F.v[1 - cur][t] = F.v[cur][t] + xv;
      F.w[1 - cur][t] = F.w[cur][t] + xw;
      F.th[t] += xt;
      m[0] = fmax(fmax(absfin(xu), absfin(xv)), fmax(absfin(xw), absfin(xt)));
    } else {
      F.u[1 - cur][t] = F.u[cur][t];
      F.v[1 - cur][t] = F.v[cur][t];
      F.w[1 - cur][t] = F.w[cur][t];
    }
  }
  block_reduce<1, true>(m, smem);
  if (publish_is_last<1>(m, F.red, F.counter)) {
    double tot[1];
    reduce_partials<1, true>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) F.rec->res = tot[0];
  }
}

// Extrapolation weights along one axis for a wall condition of zero normal derivative:
// (4 f_1 - f_2)/3 at the first wall, mirrored at the second; identity inside.
__device__ __forceinline__ int wall_weights(int a, int N, int idx[2], double wt[2]) {
  if (a == 0) {
    idx[0] = 1; idx[1] = 2; wt[0] = 4.0 / 3.0; wt[1] = -1.0 / 3.0;
    return 2;
  }
  if (a == N - 1) {
    idx[0] = N - 2; idx[1] = N - 3; wt[0] = 4.0 / 3.0; wt[1] = -1.0 / 3.0;
    return 2;
  }
  idx[0] = a; wt[0] = 1.0;
  return 1;
}

// Adiabatic walls y = 0, 1 and z = 0, 1 (x interior): theta_b = (4 theta_1 - theta_2)/3 along each
// wall normal the node lies on (on the y-z edges, the product of the two). The hot and cold
// walls keep theta = 1 and theta = 0. Max |change| joins the step record.
__global__ void __launch_bounds__(kThreads) k_theta_walls(DevParams P, Fields F, int nblocks) {
  __shared__ double smem[32];
  const int N = P.N;
  const long cnt = (long)(N - 2) * N * N;   // x interior, all y, z
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double m[1] = {0.0};
  if (t < cnt) {
    const int i = 1 + (int)(t % (N - 2));
    const long r = t / (N - 2);
    const int j = (int)(r % N), k = (int)(r / N);
    if (on_wall(j, N) | on_wall(k, N)) {
      int jy[2], kz[2];
      double wy[2], wz[2];
      const int ny = wall_weights(j, N, jy, wy), nz = wall_weights(k, N, kz, wz);
      double s = 0.0;
      for (int b = 0; b < nz; ++b) {
        double sb = 0.0;
        for (int a = 0; a < ny; ++a) sb += wy[a] * F.th[node(i, jy[a], kz[b], N)];
        s += wz[b] * sb;
      }
      const long c = node(i, j, k, N);
      m[0] = absfin(s - F.th[c]);
      F.th[c] = s;
    }
  }
  block_reduce<1, true>(m, smem);
  if (publish_is_last<1>(m, F.red, F.counter)) {
    double tot[1];
    reduce_partials<1, true>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) F.rec->res = fmax(F.rec->res, tot[0]);
  }
}

// Central div V^{n+1} at interior nodes and its maximum.
__global__ void __launch_bounds__(kThreads) k_divergence(DevParams P, Fields F, int nxt,
                                                         int nblocks) {
  __shared__ double smem[32];
  const int N = P.N, ni = N - 2;
  const long cnt = (long)ni * ni * ni;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double m[1] = {0.0};
  if (t < cnt) {
    const int i = 1 + (int)(t % ni), j = 1 + (int)((t / ni) % ni), k = 1 + (int)(t / ((long)ni * ni));
    const long c = node(i, j, k, N), sy = N, sz = (long)N * N;
    const double* u = F.u[nxt];
    const double* v = F.v[nxt];
    const double* w = F.w[nxt];
    const double d = ((u[c + 1] - u[c - 1]) + (v[c + sy] - v[c - sy]) + (w[c + sz] - w[c - sz])) *
                     (0.5 / P.h);
    F.div[c] = d;
    m[0] = absfin(d);
  }
  block_reduce<1, true>(m, smem);
  if (publish_is_last<1>(m, F.red, F.counter)) {
    double tot[1];
    reduce_partials<1, true>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) F.rec->div_max = tot[0];
  }
}

// p <- p - lambda div V at interior nodes when max|div V| > tol_div (Sec. 2.2).
__global__ void __launch_bounds__(kThreads) k_pressure_correct(DevParams P, Fields F) {
  const int N = P.N, ni = N - 2;
  const long cnt = (long)ni * ni * ni;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  if (!(F.rec->div_max > P.tol_div)) return;
  const int i = 1 + (int)(t % ni), j = 1 + (int)((t / ni) % ni), k = 1 + (int)(t / ((long)ni * ni));
  const long c = node(i, j, k, N);
  F.p[c] -= P.lambda * F.div[c];
}

// Zero normal pressure gradient on every wall: p_b = (4 p_1 - p_2)/3 along each wall normal the
// node lies on (products on edges and corners); applied after a correction.
__global__ void __launch_bounds__(kThreads) k_pressure_walls(DevParams P, Fields F) {
  const int N = P.N;
  const long n3 = (long)N * N * N;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  if (!(F.rec->div_max > P.tol_div)) return;
  const int i = (int)(t % N), j = (int)((t / N) % N), k = (int)(t / ((long)N * N));
  if (!(on_wall(i, N) | on_wall(j, N) | on_wall(k, N))) return;
  int ix[2], jy[2], kz[2];
  double wx[2], wy[2], wz[2];
  const int nx = wall_weights(i, N, ix, wx), ny = wall_weights(j, N, jy, wy),
            nz = wall_weights(k, N, kz, wz);
  double s = 0.0;
  for (int c3 = 0; c3 < nz; ++c3) {
    double s2 = 0.0;
    for (int b = 0; b < ny; ++b) {
      double s1 = 0.0;
      for (int a = 0; a < nx; ++a) s1 += wx[a] * F.p[node(ix[a], jy[b], kz[c3], N)];
      s2 += wy[b] * s1;
    }
    s += wz[c3] * s2;
  }
  F.p[t] = s;
}

// Step record: Krylov outcomes and the overall status.
__global__ void k_finish_record(Fields F) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  StepRecord* r = F.rec;
  int st = HOSC_OK;
  double lres = 0.0;
  for (int s = 0; s < 4; ++s) {
    r->iters[s] = F.ks[s].iters;
    r->lin_status[s] = F.ks[s].status;
    if (F.ks[s].status != 0) st = HOSC_ENOCONV;
    const double q = F.ks[s].r0norm > 0.0 ? F.ks[s].rnorm / F.ks[s].r0norm : 0.0;
    lres = fmax(lres, isfinite(q) ? q : INFINITY);
  }
  r->lin_res = lres;
  if (!isfinite(r->res) || !isfinite(r->div_max) || !isfinite(lres)) st = HOSC_EDIVERGED;
  r->status = st;
}

}  // namespace

int red_blocks(long count) { return (int)((count + kThreads - 1) / kThreads); }

void launch_viscosity(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long n3 = (long)P.N * P.N * P.N;
  k_viscosity<<<red_blocks(n3), kThreads, 0, s>>>(P, F.u[cur], F.v[cur], F.w[cur], F.eta, F.L[cur]);
}

void launch_sources(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long n3 = (long)P.N * P.N * P.N;
  k_sources<<<red_blocks(n3), kThreads, 0, s>>>(P, F.u[cur], F.v[cur], F.w[cur], F.th, F.p, F.eta,
                                                F.Eu[cur], F.Ev[cur], F.Ew[cur]);
}

void launch_rhs(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long ni = P.N - 2;
  const int o = 1 - cur;
  k_rhs<<<red_blocks(ni * ni * ni), kThreads, 0, s>>>(
      P, F.u[cur], F.v[cur], F.w[cur], F.th, F.L[cur], F.Eu[cur], F.Ev[cur], F.Ew[cur], F.L[o],
      F.u[o], F.v[o], F.w[o], F.Eu[o], F.Ev[o], F.Ew[o], F);
}

void launch_update(const DevParams& P, const Fields& F, int cur, cudaStream_t s) {
  const long N = P.N, n3 = N * N * N, ni = N - 2;
  const int b_all = red_blocks(n3);
  k_apply_increment<<<b_all, kThreads, 0, s>>>(P, F, cur, b_all);
  const int b_walls = red_blocks((N - 2) * N * N);
  k_theta_walls<<<b_walls, kThreads, 0, s>>>(P, F, b_walls);
  const int b_int = red_blocks(ni * ni * ni);
  k_divergence<<<b_int, kThreads, 0, s>>>(P, F, 1 - cur, b_int);
  k_pressure_correct<<<b_int, kThreads, 0, s>>>(P, F);
  k_pressure_walls<<<b_all, kThreads, 0, s>>>(P, F);
  k_finish_record<<<1, 32, 0, s>>>(F);
}

}  // namespace hosc
