// Device code of the step kernels other than the Krylov solver: S1 viscosity, S2 momentum sources,
// S3/S4 compact right-hand sides and operator weights, S6-S8 increments, wall conditions,
// divergence, pressure correction, the step record, and the float state copies (Punia & Ray,
// arXiv:2411.06563, Sec. 2.2). Each kernel is a device body taking its (virtual) block index, so
// that the one-launch-per-kernel path (hosc_step.cu) and the persistent round kernel of the pool
// (hosc_round.cu) run the same code; the __global__ wrappers launch one block per index.
//
// Layout: every field is N^3 doubles, x fastest (node (i,j,k) at i + N*(j + N*k)). One thread per
// node; node-linear thread indexing keeps consecutive threads on consecutive x.
#pragma once

#include <math.h>

#include "hosc_device.cuh"
#include "hosc_internal.h"

namespace hosc {

namespace {

// |x|, or +inf when x is not finite, on the integer units (see max_nonneg).
__device__ __forceinline__ double absfin(double x) {
  const long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return b < 0x7ff0000000000000LL ? __longlong_as_double(b) : INFINITY;
}
__device__ __forceinline__ float absfinf(float x) {
  const int b = __float_as_int(x) & 0x7fffffff;
  return b < 0x7f800000 ? __int_as_float(b) : INFINITY;
}
__device__ __forceinline__ int inward(int a, int N) { return a == 0 ? 1 : (a == N - 1 ? N - 2 : a); }
__device__ __forceinline__ int on_wall(int a, int N) { return (a == 0) | (a == N - 1); }

// Arithmetic type helpers: the sweeps run in T = double (FP64 path, mixed-precision defect
// steps) or T = float (mixed-precision sweeps: the double state is rounded to float as it is
// loaded; the rounding noise this leaves in the right-hand side is what the FP64 defect sweeps
// remove near the steady state).
template <class T> __device__ __forceinline__ T tpow(T x, T y);
template <> __device__ __forceinline__ double tpow<double>(double x, double y) { return pow(x, y); }
template <> __device__ __forceinline__ float tpow<float>(float x, float y) { return powf(x, y); }


// A scalar parameter in the arithmetic type T: the double, or its float copy made on the host.
template <class T>
__device__ __forceinline__ T par(double d, float f) {
  if constexpr (sizeof(T) == sizeof(float)) return f;
  else return d;
}

template <class T, class S>
__device__ __forceinline__ T grad_axis_t(const S* HOSC_RESTRICT f, long c, int a, int N, long st,
                                         T inv2h) {
  if (a == 0) return (T(-3) * (T)f[c] + T(4) * (T)f[c + st] - (T)f[c + 2 * st]) * inv2h;
  if (a == N - 1) return (T(3) * (T)f[c] - T(4) * (T)f[c - st] + (T)f[c - 2 * st]) * inv2h;
  return ((T)f[c + st] - (T)f[c - st]) * inv2h;
}

template <class T>
struct Grad9T {
  T ux, uy, uz, vx, vy, vz, wx, wy, wz;
};

// Spacing constants of the directions x, y, z in the arithmetic type T (spacings h, k, l of a
// box 1 x Ly x Lz; all equal in the cube): 1/(2 h_d), 1/h_d^2, h_d^2/12, 1/h_d, the edge-group
// factors and the weights of p1, q1, r1 (DevParams).
template <class T>
struct Spc {
  T i2[3], isq[3], s12[3], ih[3], grp[3], pw[6], s3;
};

template <class T>
__device__ __forceinline__ Spc<T> spacing(const DevParams& P) {
  Spc<T> s;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if constexpr (sizeof(T) == sizeof(float)) {
      s.i2[a] = P.inv2f[a];
      s.isq[a] = P.isqf[a];
      s.s12[a] = P.sq12f[a];
      s.ih[a] = P.ihf[a];
      s.grp[a] = P.grpf[a];
    } else {
      s.i2[a] = P.inv2[a];
      s.isq[a] = P.isq[a];
      s.s12[a] = P.sq12[a];
      s.ih[a] = P.ih[a];
      s.grp[a] = P.grp[a];
    }
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if constexpr (sizeof(T) == sizeof(float)) s.pw[q] = P.pwf[q];
    else s.pw[q] = P.pw[q];
  }
  if constexpr (sizeof(T) == sizeof(float)) s.s3 = P.s3f;
  else s.s3 = P.s3;
  return s;
}

template <class T, class S>
__device__ __forceinline__ Grad9T<T> velocity_gradients_t(const S* HOSC_RESTRICT u,
                                                          const S* HOSC_RESTRICT v,
                                                          const S* HOSC_RESTRICT w, int i,
                                                          int j, int k, int N,
                                                          const T i2[3]) {
  const long c = node(i, j, k, N);
  const long sy = N, sz = (long)N * N;
  Grad9T<T> g;
  g.ux = grad_axis_t<T>(u, c, i, N, 1, i2[0]);
  g.uy = grad_axis_t<T>(u, c, j, N, sy, i2[1]);
  g.uz = grad_axis_t<T>(u, c, k, N, sz, i2[2]);
  g.vx = grad_axis_t<T>(v, c, i, N, 1, i2[0]);
  g.vy = grad_axis_t<T>(v, c, j, N, sy, i2[1]);
  g.vz = grad_axis_t<T>(v, c, k, N, sz, i2[2]);
  g.wx = grad_axis_t<T>(w, c, i, N, 1, i2[0]);
  g.wy = grad_axis_t<T>(w, c, j, N, sy, i2[1]);
  g.wz = grad_axis_t<T>(w, c, k, N, sz, i2[2]);
  return g;
}

// ------------------------------------------------------------------------------------ S1

// eta = (I2 + eps)^((n-1)/2) (Eqs. 7-8), eta == 1 for n == 1; L = 1/(Pr eta) (Sec. 2.2 momentum
// coefficients). On cube edges and corners, where the one-sided strain rates of two or three
// no-slip walls vanish identically, I2 is taken at the node one step inward along each of those
// wall normals.
template <class T>
__device__ __forceinline__ void k_viscosity_body(const DevParams& P, const T* HOSC_RESTRICT u,
                                                 const T* HOSC_RESTRICT v, const T* HOSC_RESTRICT w,
                                                 T* HOSC_RESTRICT eta, T* HOSC_RESTRICT L,
                                                 const int* HOSC_RESTRICT halt, unsigned vbx) {
  const unsigned N = P.N;
  const unsigned t = vbx * blockDim.x + threadIdx.x;
  if (t >= N * N * N || *halt) return;
  const unsigned q = t / N;
  int i = (int)(t - q * N), j = (int)(q % N), k = (int)(q / N);
  T e = T(1);
  if (!P.newtonian) {
    if (on_wall(i, (int)N) + on_wall(j, (int)N) + on_wall(k, (int)N) >= 2) {
      i = inward(i, (int)N);
      j = inward(j, (int)N);
      k = inward(k, (int)N);
    }
    const Grad9T<T> g = velocity_gradients_t<T, T>(u, v, w, i, j, k, N, spacing<T>(P).i2);
    const T a = g.uz + g.wx, b = g.uy + g.vx, c = g.vz + g.wy;
    const T I2 = T(2) * (g.ux * g.ux + g.vy * g.vy + g.wz * g.wz) + a * a + b * b + c * c;
    e = tpow<T>(I2 + par<T>(P.I2_eps, P.I2_epsf), par<T>(P.eta_exp, P.eta_expf));
  }
  eta[t] = e;
  L[t] = T(1) / (par<T>(P.Pr, P.Prf) * e);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_viscosity(DevParams P, const T* HOSC_RESTRICT u,
                                                        const T* HOSC_RESTRICT v,
                                                        const T* HOSC_RESTRICT w,
                                                        T* HOSC_RESTRICT eta, T* HOSC_RESTRICT L,
                                                        const int* HOSC_RESTRICT halt) {
  k_viscosity_body(P, u, v, w, eta, L, halt, blockIdx.x);
}

// ------------------------------------------------------------------------------------ S2

// E* of the x, y, z momentum equations: the conservative momentum equations divided through by
// Pr eta so that L = 1/(Pr eta):
//   E*_x = -p_x/(Pr eta) + (2/eta)(eps_xx eta_x + eps_yx eta_y + eps_zx eta_z)
//   E*_y = -p_y/(Pr eta) + (2/eta)(eps_xy eta_x + eps_yy eta_y + eps_zy eta_z) + Ra (theta - theta_ref)/eta
//   E*_z = -p_z/(Pr eta) + (2/eta)(eps_xz eta_x + eps_yz eta_y + eps_zz eta_z)
// Gradients are central inside and one-sided at wall nodes.
template <class T>
__device__ __forceinline__ void k_sources_body(const DevParams& P, const T* HOSC_RESTRICT u,
                                               const T* HOSC_RESTRICT v, const T* HOSC_RESTRICT w,
                                               const T* HOSC_RESTRICT th, const T* HOSC_RESTRICT p,
                                               const T* HOSC_RESTRICT eta, T* HOSC_RESTRICT Eu,
                                               T* HOSC_RESTRICT Ev, T* HOSC_RESTRICT Ew,
                                               const int* HOSC_RESTRICT halt, unsigned vbx) {
  const int N = P.N;
  const unsigned t = vbx * blockDim.x + threadIdx.x;
  if (t >= (unsigned)N * N * N || *halt) return;
  const unsigned q = t / (unsigned)N;
  const int i = (int)(t - q * (unsigned)N), j = (int)(q % (unsigned)N), k = (int)(q / (unsigned)N);
  const Spc<T> sp = spacing<T>(P);
  const long sy = N, sz = (long)N * N;
  const Grad9T<T> g = velocity_gradients_t<T, T>(u, v, w, i, j, k, N, sp.i2);
  const T ex = grad_axis_t<T>(eta, t, i, N, 1, sp.i2[0]);
  const T ey = grad_axis_t<T>(eta, t, j, N, sy, sp.i2[1]);
  const T ez = grad_axis_t<T>(eta, t, k, N, sz, sp.i2[2]);
  const T px = grad_axis_t<T>(p, t, i, N, 1, sp.i2[0]);
  const T py = grad_axis_t<T>(p, t, j, N, sy, sp.i2[1]);
  const T pz = grad_axis_t<T>(p, t, k, N, sz, sp.i2[2]);
  const T e = eta[t];
  const T exy = T(0.5) * (g.uy + g.vx), exz = T(0.5) * (g.uz + g.wx), eyz = T(0.5) * (g.vz + g.wy);
  const T ie = T(1) / e;   // one division per node
  const T a = ie * par<T>(P.iPr, P.iPrf), b = T(2) * ie;
  Eu[t] = -px * a + b * (g.ux * ex + exy * ey + exz * ez);
  Ev[t] = -py * a + b * (exy * ex + g.vy * ey + eyz * ez) +
          par<T>(P.Ra, P.Raf) * ((T)th[t] - par<T>(P.theta_ref, P.theta_reff)) / e;
  Ew[t] = -pz * a + b * (exz * ex + eyz * ey + g.wz * ez);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_sources(DevParams P, const T* HOSC_RESTRICT u,
                                                     const T* HOSC_RESTRICT v,
                                                     const T* HOSC_RESTRICT w,
                                                     const T* HOSC_RESTRICT th,
                                                     const T* HOSC_RESTRICT p,
                                                     const T* HOSC_RESTRICT eta,
                                                     T* HOSC_RESTRICT Eu, T* HOSC_RESTRICT Ev,
                                                     T* HOSC_RESTRICT Ew,
                                                     const int* HOSC_RESTRICT halt) {
  k_sources_body(P, u, v, w, th, p, eta, Eu, Ev, Ew, halt, blockIdx.x);
}

// ------------------------------------------------------------------------------------ S3/S4

// 7-point neighbourhood order: centre, x+, x-, y+, y-, z+, z-.
template <class T>
struct D7 {
  T dx, dy, dz, dxx, dyy, dzz;
};

template <class T>
__device__ __forceinline__ D7<T> diffs7(const T f[7], const Spc<T>& s) {
  D7<T> d;
  d.dx = (f[1] - f[2]) * s.i2[0];
  d.dy = (f[3] - f[4]) * s.i2[1];
  d.dz = (f[5] - f[6]) * s.i2[2];
  d.dxx = (f[1] - T(2) * f[0] + f[2]) * s.isq[0];
  d.dyy = (f[3] - T(2) * f[0] + f[4]) * s.isq[1];
  d.dzz = (f[5] - T(2) * f[0] + f[6]) * s.isq[2];
  return d;
}

template <class T, class S>
__device__ __forceinline__ void load7(const S* HOSC_RESTRICT a, long c, long sy, long sz, T f[7]) {
  f[0] = (T)a[c];
  f[1] = (T)a[c + 1];
  f[2] = (T)a[c - 1];
  f[3] = (T)a[c + sy];
  f[4] = (T)a[c - sy];
  f[5] = (T)a[c + sz];
  f[6] = (T)a[c - sz];
}

// 19-point neighbourhood: 0 c, 1 x+, 2 x-, 3 y+, 4 y-, 5 z+, 6 z-,
// 7 x+y+, 8 x-y+, 9 x+y-, 10 x-y-, 11 y+z+, 12 y-z+, 13 y+z-, 14 y-z-,
// 15 z+x+, 16 z-x+, 17 z+x-, 18 z-x-.
template <class T>
__device__ __forceinline__ void load19(const T* HOSC_RESTRICT a, long c, long sy, long sz,
                                       T f[19]) {
  load7<T, T>(a, c, sy, sz, f);
  f[7] = (T)a[c + 1 + sy];
  f[8] = (T)a[c - 1 + sy];
  f[9] = (T)a[c + 1 - sy];
  f[10] = (T)a[c - 1 - sy];
  f[11] = (T)a[c + sy + sz];
  f[12] = (T)a[c - sy + sz];
  f[13] = (T)a[c + sy - sz];
  f[14] = (T)a[c - sy - sz];
  f[15] = (T)a[c + sz + 1];
  f[16] = (T)a[c - sz + 1];
  f[17] = (T)a[c + sz - 1];
  f[18] = (T)a[c - sz - 1];
}

// One edge group of Eq. (5), directions (a, b) with inverse spacings ia, ib:
//   da^2 db^2 chi - Vb da^2 db chi - Va da db^2 chi - c1 da db chi
// from F[pp], F[0p], F[mp], F[p0], F[00], F[m0], F[pm], F[0m], F[mm] (first index along a).
template <class T>
__device__ __forceinline__ T edge_group(T Fpp, T F0p, T Fmp, T Fp0, T F00, T Fm0, T Fpm, T F0m,
                                        T Fmm, T Va, T Vb, T c1, T ia, T ib) {
  const T ia2 = ia * ia, ib2 = ib * ib;
  const T d22 = (Fpp + Fmp + Fpm + Fmm - T(2) * (F0p + F0m + Fp0 + Fm0) + T(4) * F00) * ia2 * ib2;
  const T d21 = ((Fpp - T(2) * F0p + Fmp) - (Fpm - T(2) * F0m + Fmm)) * (T(0.5) * ia2 * ib);
  const T d12 = ((Fpp - T(2) * Fp0 + Fpm) - (Fmp - T(2) * Fm0 + Fmm)) * (T(0.5) * ia * ib2);
  const T d11 = (Fpp - Fmp - Fpm + Fmm) * (T(0.25) * ia * ib);
  return d22 - Vb * d21 - Va * d12 - c1 * d11;
}

// Coefficients of Eq. (5) shared by the systems with the same G*, H*, I* (K* = 0).
template <class T>
struct Eq5 {
  T G, H, I, al, be, ga, M1, M2, M3, p1, q1, r1;
};

// [1 + (dx^2 - G dx) h^2/12 + (dy^2 - H dy) k^2/12 + (dz^2 - I dz) l^2/12 + (dt/2) dt^-] f
template <class T>
__device__ __forceinline__ T bracket(const D7<T>& d, T f0, T f_prev, const Eq5<T>& c,
                                     const Spc<T>& s) {
  return f0 + s.s12[0] * (d.dxx - c.G * d.dx) + s.s12[1] * (d.dyy - c.H * d.dy) +
         s.s12[2] * (d.dzz - c.I * d.dz) + T(0.5) * (f0 - f_prev);
}

template <class T>
__device__ __forceinline__ Eq5<T> eq5_coefficients(const T G7[7], const T H7[7], const T I7[7],
                                                   T Gp, T Hp, T Ip, const Spc<T>& s) {
  Eq5<T> c;
  c.G = G7[0];
  c.H = H7[0];
  c.I = I7[0];
  const D7<T> dG = diffs7<T>(G7, s), dH = diffs7<T>(H7, s), dI = diffs7<T>(I7, s);
  c.al = T(1) + s.s12[0] * (c.G * c.G - T(2) * dG.dx);
  c.be = T(1) + s.s12[1] * (c.H * c.H - T(2) * dH.dy);
  c.ga = T(1) + s.s12[2] * (c.I * c.I - T(2) * dI.dz);
  c.M1 = bracket<T>(dG, G7[0], Gp, c, s);
  c.M2 = bracket<T>(dH, H7[0], Hp, c, s);
  c.M3 = bracket<T>(dI, I7[0], Ip, c, s);
  // p1 = -G H + 2/(h^2+k^2) (k^2 dy G + h^2 dx H), and cyclically
  c.p1 = -c.G * c.H + s.pw[0] * dG.dy + s.pw[1] * dH.dx;
  c.q1 = -c.H * c.I + s.pw[2] * dH.dz + s.pw[3] * dI.dy;
  c.r1 = -c.I * c.G + s.pw[4] * dI.dx + s.pw[5] * dG.dz;
  return c;
}

// The level-n operator of Eq. (5) applied to chi (19 points):
//  -al dx^2 - be dy^2 - ga dz^2 + M1 dx + M2 dy + M3 dz
//  - (h^2+k^2)/12 [xy group] - (k^2+l^2)/12 [yz group] - (l^2+h^2)/12 [zx group]
template <class T>
__device__ __forceinline__ T applyB(const Eq5<T>& c, const T f[19], const Spc<T>& s) {
  const D7<T> d = diffs7<T>(f, s);
  const T gxy = edge_group<T>(f[7], f[3], f[8], f[1], f[0], f[2], f[9], f[4], f[10], c.G, c.H,
                              c.p1, s.ih[0], s.ih[1]);
  const T gyz = edge_group<T>(f[11], f[5], f[12], f[3], f[0], f[4], f[13], f[6], f[14], c.H, c.I,
                              c.q1, s.ih[1], s.ih[2]);
  const T gzx = edge_group<T>(f[15], f[1], f[16], f[5], f[0], f[6], f[17], f[2], f[18], c.I, c.G,
                              c.r1, s.ih[2], s.ih[0]);
  return -c.al * d.dxx - c.be * d.dyy - c.ga * d.dzz + c.M1 * d.dx + c.M2 * d.dy + c.M3 * d.dz -
         s.grp[1] * gyz - s.grp[0] * gxy - s.grp[2] * gzx;
}

// Diagonal pseudo-time mass where the cell Reynolds number is high: the level-n operator carries
// (h_d^2/12)|G*|^2 delta^2 explicitly, and for the grid mode alternating in all three directions
// the level-(n+1) operator is only 2 dt (1/h^2 + 1/k^2 + 1/l^2) = 6 dt s3, so that mode grows once
// |G*|^2 > 24 s3 (and the mode alternating in one direction once dt |G*|^2 > 4 L). Zero in
// resolved flows; it changes the pseudo-time path only, never the steady state.
template <class T>
__device__ __forceinline__ T pseudo_time_mass(T G, T H, T I, T L, T dt, T s3, T kappa) {
  const T g2 = G * G + H * H + I * I;
  const T s = fmax(T(0), fmax(dt * (g2 / T(6) - s3), dt * g2 / T(6) - T(2) * L / T(3)));
  return kappa * s;
}

// Right-hand sides of the increment form of Eq. (6),  A (chi^{n+1} - chi^n) = dt (R - B chi^n),
// for u, v, w, theta at interior nodes, and the seven level-(n+1) weights L1..L7 of the momentum
// and energy systems. Tc: arithmetic and the type of L, E*; Ts: type of the outputs.
template <class Tc, class Ts>
// The float build is bounded to 80 registers (three 256-thread blocks per SM); the double builds
// keep the compiler's choice.
__device__ __forceinline__ void k_rhs_body(const DevParams& P, const Tc* HOSC_RESTRICT u,
                                           const Tc* HOSC_RESTRICT v, const Tc* HOSC_RESTRICT w,
                                           const Tc* HOSC_RESTRICT th, const Tc* HOSC_RESTRICT L,
                                           const Tc* HOSC_RESTRICT Eu, const Tc* HOSC_RESTRICT Ev,
                                           const Tc* HOSC_RESTRICT Ew, const Tc* HOSC_RESTRICT Lp,
                                           const Tc* HOSC_RESTRICT up, const Tc* HOSC_RESTRICT vp,
                                           const Tc* HOSC_RESTRICT wp, const Tc* HOSC_RESTRICT Eup,
                                           const Tc* HOSC_RESTRICT Evp, const Tc* HOSC_RESTRICT Ewp,
                                           const Fields& F, unsigned vbx) {
  const int N = P.N;
  const unsigned ni = N - 2;
  const unsigned t = vbx * blockDim.x + threadIdx.x;
  if (t >= ni * ni * ni || *F.halt) return;
  const unsigned q = t / ni;
  const int i = 1 + (int)(t - q * ni), j = 1 + (int)(q % ni), k = 1 + (int)(q / ni);
  const long sy = N, sz = (long)N * N;
  const long c = node(i, j, k, N);
  const Spc<Tc> sp = spacing<Tc>(P);
  const Tc tdt = par<Tc>(P.dt, P.dtf);
  Tc rv[4], Am[7], Ae[7];   // right-hand sides and weights, stored at the end

  Tc L7[7], u7[7], v7[7], w7[7];
  load7<Tc, Tc>(L, c, sy, sz, L7);
  load7<Tc, Tc>(u, c, sy, sz, u7);
  load7<Tc, Tc>(v, c, sy, sz, v7);
  load7<Tc, Tc>(w, c, sy, sz, w7);
  const Tc Lc = L7[0];
  const Tc Lpc = P.have_prev ? Lp[c] : Lc;
  const Tc upc = P.have_prev ? (Tc)up[c] : u7[0];
  const Tc vpc = P.have_prev ? (Tc)vp[c] : v7[0];
  const Tc wpc = P.have_prev ? (Tc)wp[c] : w7[0];

  // ---------------- momentum: L = 1/(Pr eta), G* = u L, H* = v L, I* = w L, K* = 0
  {
    Tc G7[7], H7[7], I7[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      G7[q] = u7[q] * L7[q];
      H7[q] = v7[q] * L7[q];
      I7[q] = w7[q] * L7[q];
    }
    const Eq5<Tc> cm = eq5_coefficients<Tc>(G7, H7, I7, upc * Lpc, vpc * Lpc, wpc * Lpc, sp);
    // one momentum system: source E (level n, and n-1 when kept) and the field X
    auto system = [&](const Tc* HOSC_RESTRICT E, const Tc* HOSC_RESTRICT Ep,
                      const Tc* HOSC_RESTRICT X) {
      Tc E7[7], f19[19];
      load7<Tc, Tc>(E, c, sy, sz, E7);
      const Tc Epc = P.have_prev ? Ep[c] : E7[0];
      const Tc R = bracket<Tc>(diffs7<Tc>(E7, sp), E7[0], Epc, cm, sp);
      load19<Tc>(X, c, sy, sz, f19);
      return tdt * (R - applyB<Tc>(cm, f19, sp));
    };
    rv[0] = system(Eu, Eup, u);
    rv[1] = system(Ev, Evp, v);
    rv[2] = system(Ew, Ewp, w);
    // level-(n+1) weights (Eq. 6): M_d = -dt/(2L) + h_d^2/12, M15 = (h^2/(6L)) dx L, ...
    const D7<Tc> dL = diffs7<Tc>(L7, sp);
    const Tc iL = Tc(1) / Lc;   // one division per node
    const Tc m0 = Tc(-0.5) * tdt * iL, inv6L = Tc(2) * iL;   // h_d^2/(6L) = (h_d^2/12) (2/L)
    const Tc Mx = m0 + sp.s12[0], My = m0 + sp.s12[1], Mz = m0 + sp.s12[2];
    const Tc m15 = sp.s12[0] * inv6L * dL.dx, m16 = sp.s12[1] * inv6L * dL.dy,
             m17 = sp.s12[2] * inv6L * dL.dz;
    Tc M18 = Tc(0.5) * (Lc - Lpc) + sp.s12[0] * (dL.dxx - cm.G * dL.dx) +
             sp.s12[1] * (dL.dyy - cm.H * dL.dy) + sp.s12[2] * (dL.dzz - cm.I * dL.dz);
    // keep the extrapolated mass positive where L changes fast (the steady state is unaffected)
    const Tc alim = par<Tc>(P.a_limit, P.a_limitf), kap = par<Tc>(P.a_boost, P.a_boostf);
    if (alim > Tc(0)) M18 = fmax(M18, -alim * Lc);
    const Tc sig_m =
        kap > Tc(0) ? pseudo_time_mass<Tc>(cm.G, cm.H, cm.I, Lc, tdt, sp.s3, kap) : Tc(0);
    const Tc ax = Mx * sp.isq[0], ay = My * sp.isq[1], az = Mz * sp.isq[2];
    Am[0] = Lc * (Tc(1) - Tc(2) * (ax + ay + az)) + M18 + sig_m;
    Am[1] = Lc * (ax - Mx * cm.G * sp.i2[0] + m15 * sp.i2[0]);
    Am[2] = Lc * (ax + Mx * cm.G * sp.i2[0] - m15 * sp.i2[0]);
    Am[3] = Lc * (ay - My * cm.H * sp.i2[1] + m16 * sp.i2[1]);
    Am[4] = Lc * (ay + My * cm.H * sp.i2[1] - m16 * sp.i2[1]);
    Am[5] = Lc * (az - Mz * cm.I * sp.i2[2] + m17 * sp.i2[2]);
    Am[6] = Lc * (az + Mz * cm.I * sp.i2[2] - m17 * sp.i2[2]);
  }
  // ---------------- energy: L = 1, G* = u, H* = v, I* = w, K* = E* = 0
  {
    const Eq5<Tc> ce = eq5_coefficients<Tc>(u7, v7, w7, upc, vpc, wpc, sp);
    Tc f19[19];
    load19<Tc>(th, c, sy, sz, f19);
    rv[3] = -tdt * applyB<Tc>(ce, f19, sp);
    const Tc m0 = Tc(-0.5) * tdt;
    const Tc Mx = m0 + sp.s12[0], My = m0 + sp.s12[1], Mz = m0 + sp.s12[2];
    const Tc ax = Mx * sp.isq[0], ay = My * sp.isq[1], az = Mz * sp.isq[2];
    const Tc kap = par<Tc>(P.a_boost, P.a_boostf);
    const Tc sig_e =
        kap > Tc(0) ? pseudo_time_mass<Tc>(ce.G, ce.H, ce.I, Tc(1), tdt, sp.s3, kap) : Tc(0);
    Ae[0] = Tc(1) - Tc(2) * (ax + ay + az) + sig_e;
    Ae[1] = ax - Mx * ce.G * sp.i2[0];
    Ae[2] = ax + Mx * ce.G * sp.i2[0];
    Ae[3] = ay - My * ce.H * sp.i2[1];
    Ae[4] = ay + My * ce.H * sp.i2[1];
    Ae[5] = az - Mz * ce.I * sp.i2[2];
    Ae[6] = az + Mz * ce.I * sp.i2[2];
  }
  if (P.precond) {   // Jacobi row scaling: each right-hand side over its row's diagonal
    const Tc dm = Am[0] != Tc(0) ? Am[0] : Tc(1), de = Ae[0] != Tc(0) ? Ae[0] : Tc(1);
#pragma unroll
    for (int s = 0; s < 3; ++s) rv[s] /= dm;
    rv[3] /= de;
    if constexpr (sizeof(Ts) != sizeof(float)) {   // the planar weights too (the compact float
#pragma unroll                                      // operators divide by D when applied)
      for (int q = 0; q < 7; ++q) {
        Am[q] /= dm;
        Ae[q] /= de;
      }
    }
  }
  if constexpr (sizeof(Ts) == sizeof(float)) {   // interleaved float storage
    F.kr0[c] = make_float4((float)rv[0], (float)rv[1], (float)rv[2], (float)rv[3]);
    // compact operators: the antisymmetric halves (W_{-d} - W_{+d})/2 and the diagonal
    F.kwm[c] = make_float4((float)(Tc(0.5) * (Am[2] - Am[1])), (float)(Tc(0.5) * (Am[4] - Am[3])),
                           (float)(Tc(0.5) * (Am[6] - Am[5])), (float)Am[0]);
    F.kwe[c] = make_float4((float)(Tc(0.5) * (Ae[2] - Ae[1])), (float)(Tc(0.5) * (Ae[4] - Ae[3])),
                           (float)(Tc(0.5) * (Ae[6] - Ae[5])), (float)Ae[0]);
    F.kL[c] = (float)Lc;
  } else {                                         // planar double storage
#pragma unroll
    for (int s = 0; s < 4; ++s) F.rhs[s][c] = (double)rv[s];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      F.Am[q][c] = (double)Am[q];
      F.Ae[q][c] = (double)Ae[q];
    }
  }
}

template <class Tc, class Ts>
__global__ void __launch_bounds__(kThreads, sizeof(Tc) == sizeof(float) ? 3 : 0) k_rhs(
    DevParams P, const Tc* HOSC_RESTRICT u, const Tc* HOSC_RESTRICT v,
    const Tc* HOSC_RESTRICT w, const Tc* HOSC_RESTRICT th, const Tc* HOSC_RESTRICT L,
    const Tc* HOSC_RESTRICT Eu, const Tc* HOSC_RESTRICT Ev, const Tc* HOSC_RESTRICT Ew,
    const Tc* HOSC_RESTRICT Lp, const Tc* HOSC_RESTRICT up, const Tc* HOSC_RESTRICT vp,
    const Tc* HOSC_RESTRICT wp, const Tc* HOSC_RESTRICT Eup, const Tc* HOSC_RESTRICT Evp,
    const Tc* HOSC_RESTRICT Ewp, Fields F) {
  k_rhs_body<Tc, Ts>(P, u, v, w, th, L, Eu, Ev, Ew, Lp, up, vp, wp, Eup, Evp, Ewp, F,
                     blockIdx.x);
}

// ------------------------------------------------------------------------------------ S6-S8

// chi^{n+1} = chi^n + x at interior nodes (u, v, w into the other buffer, theta in place); wall
// velocities are carried over. Max |x| over the four systems goes to the step record.
template <class Ts>
__device__ __forceinline__ void k_apply_increment_body(const DevParams& P, const Fields& F,
                                                       int cur, int nblocks, unsigned vbx) {
  __shared__ double smem[64];
  if (*F.halt) return;
  const unsigned N = P.N;
  const unsigned n3 = N * N * N;
  const unsigned t = vbx * blockDim.x + threadIdx.x;
  double m[2] = {0.0, 0.0};   // max |x| of u, v, w and of theta
  if (t < n3) {
    const unsigned q = t / N;
    const unsigned i = t - q * N, j = q % N, k = q / N;
    const bool inner = i > 0 && j > 0 && k > 0 && i < N - 1 && j < N - 1 && k < N - 1;
    if (inner) {
      double xu, xv, xw, xt;
      if constexpr (sizeof(Ts) == sizeof(float)) {   // interleaved float increments
        const float4 x4 = F.kx[t];
        xu = x4.x;
        xv = x4.y;
        xw = x4.z;
        xt = x4.w;
        // magnitudes in float (exact), widened once
        m[0] = fmaxf(fmaxf(absfinf(x4.x), absfinf(x4.y)), absfinf(x4.z));
        m[1] = absfinf(x4.w);
      } else {
        xu = F.x[0][t];
        xv = F.x[1][t];
        xw = F.x[2][t];
        xt = F.x[3][t];
        m[0] = max_nonneg(max_nonneg(absfin(xu), absfin(xv)), absfin(xw));
        m[1] = absfin(xt);
      }
      F.u[1 - cur][t] = F.u[cur][t] + xu;
      F.v[1 - cur][t] = F.v[cur][t] + xv;
      F.w[1 - cur][t] = F.w[cur][t] + xw;
      F.th[t] += xt;
    } else {
      F.u[1 - cur][t] = F.u[cur][t];
      F.v[1 - cur][t] = F.v[cur][t];
      F.w[1 - cur][t] = F.w[cur][t];
    }
  }
  block_reduce<2, true>(m, smem);
  if (publish_is_last<2>(m, F.red, F.counter, vbx, nblocks)) {
    double tot[2];
    reduce_partials<2, true>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      // an inner pressure pass changes u, v, w only: theta's change stays that of the first pass
      if (!P.inner_pass) F.rec->res_theta = tot[1];
      F.rec->res = fmax(tot[0], F.rec->res_theta);
    }
  }
}

template <class Ts>
__global__ void __launch_bounds__(kThreads) k_apply_increment(DevParams P, Fields F, int cur,
                                                              int nblocks) {
  k_apply_increment_body<Ts>(P, F, cur, nblocks, blockIdx.x);
}

__device__ __forceinline__ int node32(int i, int j, int k, int N) { return i + N * (j + N * k); }

// Node number t of the y faces (x interior, all z), then of the z faces (x, y interior):
// 0 <= t < 2 (N-2) N + 2 (N-2)^2, x fastest.
__device__ __forceinline__ void boundary_yz(int t, int N, int& i, int& j, int& k) {
  const int ni = N - 2;
  if (t < 2 * ni * N) {
    const int side = t / (ni * N), r = t - side * ni * N;
    const int q = r / ni;
    i = 1 + (r - q * ni);
    k = q;
    j = side ? N - 1 : 0;
  } else {
    const int u = t - 2 * ni * N;
    const int side = u / (ni * ni), r = u - side * ni * ni;
    const int q = r / ni;
    i = 1 + (r - q * ni);
    j = 1 + q;
    k = side ? N - 1 : 0;
  }
}

// Node number t of the cube's boundary, 0 <= t < N^3 - (N-2)^3: the x faces, then the y and z
// faces as in boundary_yz.
__device__ __forceinline__ void boundary_node(int t, int N, int& i, int& j, int& k) {
  const int N2 = N * N;
  if (t < 2 * N2) {
    const int side = t / N2, r = t - side * N2;
    const int q = r / N;
    j = r - q * N;
    k = q;
    i = side ? N - 1 : 0;
  } else {
    boundary_yz(t - 2 * N2, N, i, j, k);
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
__device__ __forceinline__ void k_theta_walls_body(const DevParams& P, const Fields& F,
                                                   int nblocks, unsigned vbx) {
  __shared__ double smem[32];
  if (*F.halt) return;
  const int N = P.N, ni = N - 2;
  const int t = vbx * blockDim.x + threadIdx.x;
  double m[1] = {0.0};
  int i, j, k;
  if (t < 2 * ni * N + 2 * ni * ni) {   // the y faces, then the z faces (x interior)
    boundary_yz(t, N, i, j, k);
    int jy[2], kz[2];
    double wy[2], wz[2];
    const int ny = wall_weights(j, N, jy, wy), nz = wall_weights(k, N, kz, wz);
    double s = 0.0;
    for (int b = 0; b < nz; ++b) {
      double sb = 0.0;
      for (int a = 0; a < ny; ++a) sb += wy[a] * F.th[node32(i, jy[a], kz[b], N)];
      s += wz[b] * sb;
    }
    const int c = node32(i, j, k, N);
    m[0] = absfin(s - F.th[c]);
    F.th[c] = s;
  }
  block_reduce<1, true>(m, smem);
  if (publish_is_last<1>(m, F.red, F.counter, vbx, nblocks)) {
    double tot[1];
    reduce_partials<1, true>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) {
      F.rec->res = fmax(F.rec->res, tot[0]);
      if (!P.inner_pass) F.rec->res_theta = fmax(F.rec->res_theta, tot[0]);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_theta_walls(DevParams P, Fields F, int nblocks) {
  k_theta_walls_body(P, F, nblocks, blockIdx.x);
}

// Central div V^{n+1} at interior nodes and its maximum.
__device__ __forceinline__ void k_divergence_body(const DevParams& P, const Fields& F, int nxt,
                                                  int nblocks, unsigned vbx) {
  __shared__ double smem[32];
  if (*F.halt) return;
  const int N = P.N, ni = N - 2;
  const int cnt = ni * ni * ni;
  const int t = vbx * blockDim.x + threadIdx.x;
  double m[1] = {0.0};
  if (t < cnt) {
    const int q = t / ni, i = 1 + (t - q * ni), j = 1 + q % ni, k = 1 + q / ni;
    const int c = node32(i, j, k, N), sy = N, sz = N * N;
    const double* u = F.u[nxt];
    const double* v = F.v[nxt];
    const double* w = F.w[nxt];
    const double d = (u[c + 1] - u[c - 1]) * P.inv2[0] + (v[c + sy] - v[c - sy]) * P.inv2[1] +
                     (w[c + sz] - w[c - sz]) * P.inv2[2];
    F.div[c] = d;
    m[0] = absfin(d);
  }
  block_reduce<1, true>(m, smem);
  if (publish_is_last<1>(m, F.red, F.counter, vbx, nblocks)) {
    double tot[1];
    reduce_partials<1, true>(tot, F.red, nblocks, F.counter, smem);
    if (threadIdx.x == 0) F.rec->div_max = tot[0];
  }
}

__global__ void __launch_bounds__(kThreads) k_divergence(DevParams P, Fields F, int nxt,
                                                         int nblocks) {
  k_divergence_body(P, F, nxt, nblocks, blockIdx.x);
}

// p <- p - lambda div V at interior nodes when max|div V| > tol_div (Sec. 2.2).
__device__ __forceinline__ void k_pressure_correct_body(const DevParams& P, const Fields& F,
                                                        unsigned vbx) {
  const int N = P.N, ni = N - 2;
  const int cnt = ni * ni * ni;
  const int t = vbx * blockDim.x + threadIdx.x;
  if (t >= cnt || *F.halt) return;
  if (!(F.rec->div_max > P.tol_div)) return;
  const int q = t / ni, i = 1 + (t - q * ni), j = 1 + q % ni, k = 1 + q / ni;
  const int c = node32(i, j, k, N);
  double lam = P.lambda;
  if (P.lambda_mode) {   // viscosity-scaled relaxation: eta of level n (float in FP32 sweeps)
    const double eta =
        P.sweep_fp32 ? (double)reinterpret_cast<const float*>(F.eta)[c] : F.eta[c];
    lam = fmin(P.lambda * eta, P.lambda_cap);
  }
  F.p[c] -= lam * F.div[c];
}

__global__ void __launch_bounds__(kThreads) k_pressure_correct(DevParams P, Fields F) {
  k_pressure_correct_body(P, F, blockIdx.x);
}

// Zero normal pressure gradient on every wall: p_b = (4 p_1 - p_2)/3 along each wall normal the
// node lies on (products on edges and corners); applied after a correction.
__device__ __forceinline__ void k_pressure_walls_body(const DevParams& P, const Fields& F,
                                                      unsigned vbx) {
  const int N = P.N, ni = N - 2;
  const int t = vbx * blockDim.x + threadIdx.x;
  if (t >= N * N * N - ni * ni * ni || *F.halt) return;
  if (!(F.rec->div_max > P.tol_div)) return;
  int i, j, k;
  boundary_node(t, N, i, j, k);
  int ix[2], jy[2], kz[2];
  double wx[2], wy[2], wz[2];
  const int nx = wall_weights(i, N, ix, wx), ny = wall_weights(j, N, jy, wy),
            nz = wall_weights(k, N, kz, wz);
  double s = 0.0;
  for (int c3 = 0; c3 < nz; ++c3) {
    double s2 = 0.0;
    for (int b = 0; b < ny; ++b) {
      double s1 = 0.0;
      for (int a = 0; a < nx; ++a) s1 += wx[a] * F.p[node32(ix[a], jy[b], kz[c3], N)];
      s2 += wy[b] * s1;
    }
    s += wz[c3] * s2;
  }
  F.p[node32(i, j, k, N)] = s;
}

__global__ void __launch_bounds__(kThreads) k_pressure_walls(DevParams P, Fields F) {
  k_pressure_walls_body(P, F, blockIdx.x);
}

// Step record: Krylov outcomes and the overall status; appended to the ring. A failed step (or,
// when asked, a steady one) halts the rest of the enqueued sequence.
__device__ __forceinline__ void k_finish_record_body(const DevParams& P, const Fields& F,
                                                     unsigned vbx) {
  if (threadIdx.x != 0 || vbx != 0) return;
  if (*F.halt) return;
  StepRecord* r = F.rec;
  int st = HOSC_OK;
  double lres = 0.0;
  for (int s = 0; s < 4; ++s) {
    r->iters[s] = F.ks[s].iters;
    r->lin_status[s] = F.ks[s].status;
    // HOSC_ECUDA: a bounded wait inside a Krylov kernel ran out; anything else: no convergence
    if (F.ks[s].status == HOSC_ECUDA) st = HOSC_ECUDA;
    else if (F.ks[s].status != 0 && st != HOSC_ECUDA) st = HOSC_ENOCONV;
    const double q = F.ks[s].r0norm > 0.0 ? F.ks[s].rnorm / F.ks[s].r0norm : 0.0;
    lres = fmax(lres, isfinite(q) ? q : INFINITY);
  }
  r->lin_res = lres;
  if (!isfinite(r->res) || !isfinite(r->div_max) || !isfinite(lres)) st = HOSC_EDIVERGED;
  r->status = st;
  const unsigned pos = *F.ring_pos;
  F.ring[pos % kRing] = *r;
  *F.ring_pos = pos + 1;
  if (st != HOSC_OK) *F.halt = 1;
  else if (*F.steady_stop && r->res < P.steady_res && r->div_max < P.div_steady) *F.halt = 2;
}

__global__ void k_finish_record(DevParams P, Fields F) {
  k_finish_record_body(P, F, blockIdx.x);
}

__global__ void k_arm(int* halt, unsigned int* ring_pos, int* steady_stop, int stop) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *halt = 0;
    *ring_pos = 0u;
    *steady_stop = stop;
  }
}

}  // namespace

namespace {
// Float copies of the state for the FP32 sweeps (one rounding per node and step).
__device__ __forceinline__ void k_shadow_body(int n3, const double* HOSC_RESTRICT u,
                                              const double* HOSC_RESTRICT v,
                                              const double* HOSC_RESTRICT w,
                                              const double* HOSC_RESTRICT th,
                                              const double* HOSC_RESTRICT p, float* HOSC_RESTRICT us,
                                              float* HOSC_RESTRICT vs, float* HOSC_RESTRICT ws,
                                              float* HOSC_RESTRICT ths, float* HOSC_RESTRICT ps,
                                              const int* HOSC_RESTRICT halt, unsigned vbx) {
  const int t = vbx * blockDim.x + threadIdx.x;
  if (t >= n3 || *halt) return;
  us[t] = (float)u[t];
  vs[t] = (float)v[t];
  ws[t] = (float)w[t];
  if (ths) {
    ths[t] = (float)th[t];
    ps[t] = (float)p[t];
  }
}

__global__ void __launch_bounds__(kThreads) k_shadow(int n3, const double* HOSC_RESTRICT u,
                                                     const double* HOSC_RESTRICT v,
                                                     const double* HOSC_RESTRICT w,
                                                     const double* HOSC_RESTRICT th,
                                                     const double* HOSC_RESTRICT p,
                                                     float* HOSC_RESTRICT us, float* HOSC_RESTRICT vs,
                                                     float* HOSC_RESTRICT ws,
                                                     float* HOSC_RESTRICT ths,
                                                     float* HOSC_RESTRICT ps,
                                                     const int* HOSC_RESTRICT halt) {
  k_shadow_body(n3, u, v, w, th, p, us, vs, ws, ths, ps, halt, blockIdx.x);
}
}  // namespace

}  // namespace hosc
