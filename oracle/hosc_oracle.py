"""Plain FP64 CPU oracle of the HOSC (19,7) scheme for 3D power-law natural convection.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference leg of ``bench.py`` may import or run this module. The CUDA library never calls it and
shares no code, table or helper with it.

What it follows (Punia & Ray, "New Higher-Order Super-Compact Finite Difference Scheme to Study
Three-Dimensional Natural Convection and Entropy Generation in Non-Newtonian Fluids",
arXiv:2411.06563):

* Sec. 2.1, Eqs. (1)-(5) of the problem statement and the conservative momentum form: the
  Boussinesq equations with the power-law stress, eta = I2^((n-1)/2) (Eqs. 6-8).
* Sec. 2.1, boundary conditions (hot wall x=0, cold wall x=1, adiabatic other walls, no slip,
  zero normal pressure gradient everywhere).
* Sec. 2.2, Eq. (1): the generic transport equation
      L chi_t + H* chi_y + G* chi_x + I* chi_z + K* chi - lap(chi) = E*.
* Sec. 2.2, Eq. (5) and its coefficient list (alpha, beta, gamma, M1..M4, R, p1, q1, r1): the
  implicit HOSC operator, written here literally as a composition of the central-difference
  operators delta_x, delta_x^2, ... acting on coefficient fields. Eq. (6) is the same scheme
  expanded into the 7 level-(n+1) and 19 level-n stencil weights (Q = A - dt*B).
* Sec. 2.2 (text after Eq. 6): momentum coefficients L=1/(Pr eta), G*=u/(Pr eta), ...; energy
  coefficients L=1, G*=u, ...; central pressure gradients inside, one-sided at boundary nodes;
  unpreconditioned BiCGSTAB; the modified artificial-compressibility correction p <- p - lam div V
  applied when max|div V| exceeds a tolerance.
* Sec. 4.2/4.3: local and average Nusselt numbers, entropy generation E_HT, E_FF, E_local,
  E_total and the Bejan number.

Readings of passages that are silent, garbled or inconsistent (each one is listed in the design
notes of the repository):

* R1  eta = (I2 + eps)^((n-1)/2) with a small regulariser eps (the paper's eta is singular at
      I2=0 for n<1); eta == 1 exactly when n == 1.
* R1b On cube edges and corners (where I2 = 0 identically) eta is copied from the node one step
      inward along each wall normal (see ``edge_from_diagonal``).
* R2  Momentum E* is the conservative momentum equation divided through by Pr*eta, consistent
      with L = 1/(Pr eta):  E*_x = -p_x/(Pr eta) + (2/eta)(eps_xx eta_x + eps_yx eta_y + eps_zx eta_z),
      and E*_y additionally + Ra (theta - theta_ref)/eta (gravity along -y).
* R3  theta_ref (Boussinesq reference temperature) is a parameter, default 1/2.
* R4  "Hybrid" BiCGSTAB = the standard (van der Vorst) BiCGSTAB, no preconditioner, started from
      the level-n field; stop when ||r_k||_2 <= tol * ||r_0||_2.
* R5  One pressure correction per time step; it is applied at interior nodes when
      max|div V| > tol_div, then the wall pressure is set from the zero-normal-gradient condition
      by second-order one-sided extrapolation p_b = (4 p_1 - p_2)/3.
* R6  The four systems (u, v, w, theta) all use level-n coefficients; wall values of chi^{n+1} in
      the level-(n+1) stencil are the level-n wall values (the adiabatic theta walls are updated
      after the solves by (4 t_1 - t_2)/3).
* R7  Wall-node derivatives (strain rates, grad eta, grad p, grad theta) are second-order
      one-sided along the wall normal, central along the wall.
* R8  delta_t^- f = (f^n - f^{n-1})/dt for the coefficient fields; it is zero at the first step.
* R9  M18 is read from the delta_t^+ bracket of Eq. (5) itself (the printed M18 line is garbled).
* R10 Nu_local = -d theta/dx at the hot wall (fourth-order one-sided), Nu_avg(z) = its mean over
      y (Simpson), Nu_max = max_z Nu_avg(z) (the quantity of Table 2), Nu_mean = surface mean.
* R11 chi* = phi* = phi (default 1e-4), so E_FF = phi * eta * I2; Be = int E_HT / int E_local.
* R12 The initial interior temperature is theta_init (default 1/2 = theta_ref): the fluid at rest
      with constant pressure is then in equilibrium with the buoyancy term at t = 0.
* R18 The diagonal part M18 of the level-(n+1) operator is limited below by -a_limit * L (default
      a_limit = 1/4) so the operator keeps a positive mass when L changes fast (see assemble_A).
* R20 use_history = 0 sets delta_t^- = 0 at every step: a first-order pseudo-time march with the
      same steady state, free of the period-2 computational mode of the three-level scheme.
* R19 Where the cell Reynolds number |G*| h is high, a diagonal pseudo-time mass is added to the
      level-(n+1) operator (see pseudo_time_mass). R18 and R19 change A only: the discrete steady
      state B chi = R of Eq. (5) is the paper's.
* R22 Optional inner pressure passes within a step (the "previous pressure iteration" of
      Sec. 2.2), see step; the default is one correction per step (R5).
* R23 A box 1 x Ly x Lz with N nodes per side (spacings h, k, l), the general form of Eqs. (5)-(6);
      the cube by default.
* R24 solver = 1: BiCGSTAB(2), the other reading of the "hybrid" BiCGSTAB (solve_bicgstab_l).
* R25 lam_mode = 1: the relaxation of the pressure correction scaled node by node with the
      level-n viscosity, lam * eta, at most 0.9 h^2/dt (see relaxation); the default is the
      paper's single lam.

Pinned readings without a printed value: R18 (the limited operator differs from the unlimited
one only on the diagonal, exactly where M18/L is below -a_limit, and both reach one steady
state), R19 (the frozen-coefficient amplification of the two highest grid modes, worked out by
hand from Eq. 5: the mass starts exactly where the unmassed amplification of the checkerboard
mode reaches zero, or where that of the one-direction mode passes -1, and keeps both within
[-1, 1]), R1b (a field whose edge strain differs from its neighbours'), R11 (E_FF in closed form
on linear fields).

Parity unpinned (no value in the paper fixes them; each sets the pseudo-time path or regularises,
and the steady state B chi = R does not depend on lambda or dt, which the steady-state pin
checks): the regulariser eps of R1 (the 9^3 steady state is the same to ten digits for eps from
1e-12 to 1e-8), the relaxation lambda and the pseudo-time step dt.

Layout: a field is a numpy array f[z, y, x] of shape (N, N, N); node (i, j, k) sits at
x = i*h, y = j*k, z = k*l with spacings h = 1/(N-1), k = Ly/(N-1), l = Lz/(N-1). The flattened
index is i + N*(j + N*k).
"""

import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Params", "Grid", "scalar_coefficients", "assemble_A", "apply_B", "solve_bicgstab",
    "solve_bicgstab_l", "solve_system", "viscosity", "momentum_sources", "initial_state", "step", "solve_steady",
    "apply_theta_bc", "apply_pressure_bc", "divergence", "diagnostics", "steady_certificate",
    "grad_full", "strain_gradients", "relaxation",
]


# --------------------------------------------------------------------------------- parameters

class Params:
    """Problem and solver parameters (Sec. 2.1 dimensionless groups; Sec. 3.1 dt = 0.02)."""

    def __init__(self, N, Ra, Pr=1.0, n=1.0, dt=0.02, lam=None, theta_ref=0.5, I2_eps=1e-10,
                 phi=1e-4, tol_div=1e-6, tol_lin=1e-12, max_lin_iter=2000, theta_init=0.5,
                 a_limit=0.25, a_boost=1.0, use_history=1, precond=0, inner_max=0, Ly=1.0,
                 Lz=1.0, solver=0, lam_mode=0):
        self.N = int(N)
        # Box 1 x Ly x Lz (lengths in units of the hot-cold wall distance) on N nodes per side:
        # spacings h = 1/(N-1), k = Ly/(N-1), l = Lz/(N-1) (the scheme of Sec. 2.2 is written
        # for unequal spacings; the paper's cavity is the cube, Ly = Lz = 1)
        self.Ly = float(Ly)
        self.Lz = float(Lz)
        self.Ra = float(Ra)
        self.Pr = float(Pr)
        self.n = float(n)
        self.dt = float(dt)
        h = min(self.spacings())
        # Relaxation of the artificial-compressibility update (not given in the paper): the
        # smaller of h^2/(4 dt) and Pr/10 (h the smallest spacing). Above h^2/dt the highest
        # grid mode of the coupled update grows even at constant viscosity; at small dt the
        # pressure mode needs lam below about twice the smallest Pr*eta.
        self.lam = float(min(0.25 * h * h / self.dt, 0.1 * self.Pr) if lam is None else lam)
        # Lower limit of M18 in units of L (reading R18); 0 disables the limiter.
        self.a_limit = float(a_limit)
        # Factor of the pseudo-time mass added where the cell Reynolds number is high (R19).
        self.a_boost = float(a_boost)
        # 1: delta_t^- from the level n-1 history (Eq. 5); 0: delta_t^- = 0 every step (R20).
        self.use_history = int(use_history)
        # 1: Jacobi row scaling of each level-(n+1) system before BiCGSTAB (not in the paper;
        # the solution is the same, only the Krylov iteration changes)
        self.precond = int(precond)
        # >= 1: up to this many inner pressure iterations per step (see step); 0: one pressure
        # correction per step
        self.inner_max = int(inner_max)
        # 0: BiCGSTAB (the reading of Sec. 2.2's solver used throughout); 1: BiCGSTAB(2)
        self.solver = int(solver)
        # Relaxation of the pressure correction (reading R25): 0 the single parameter lam of
        # Sec. 2.2; 1 lam * eta at each node (eta the level-n apparent viscosity), at most
        # 0.9 h^2/dt (h the smallest spacing)
        self.lam_mode = int(lam_mode)
        self.theta_ref = float(theta_ref)
        self.theta_init = float(theta_init)
        self.I2_eps = float(I2_eps)
        self.phi = float(phi)
        self.tol_div = float(tol_div)
        self.tol_lin = float(tol_lin)
        self.max_lin_iter = int(max_lin_iter)

    def spacings(self):
        """(h, k, l): node spacings along x, y, z."""
        m = self.N - 1
        return 1.0 / m, self.Ly / m, self.Lz / m


# --------------------------------------------------------------------------------- operators

def _d1(n, dx):
    """1D first central difference delta (Sec. 2.2, Eq. 2); rows 0 and n-1 are empty."""
    m = sp.lil_matrix((n, n))
    for i in range(1, n - 1):
        m[i, i + 1] = 1.0 / (2.0 * dx)
        m[i, i - 1] = -1.0 / (2.0 * dx)
    return m.tocsr()


def _d2(n, dx):
    """1D second central difference delta^2 (Sec. 2.2, Eq. 2); rows 0 and n-1 are empty."""
    m = sp.lil_matrix((n, n))
    for i in range(1, n - 1):
        m[i, i + 1] = 1.0 / (dx * dx)
        m[i, i] = -2.0 / (dx * dx)
        m[i, i - 1] = 1.0 / (dx * dx)
    return m.tocsr()


class Grid:
    """Uniform N^3 node grid of the box 1 x Ly x Lz (spacings h, k, l along x, y, z; the unit
    cube by default) and the central-difference operators of Eq. (2).

    Each 3D operator is an N^3 x N^3 sparse matrix acting on flattened fields. The row of a node
    is filled only where the node is interior along that operator's direction, so products such
    as delta_x^2 delta_y^2 are exact tensor-product stencils at every interior node.
    """

    def __init__(self, N, Ly=1.0, Lz=1.0):
        self.N = N = int(N)
        self.h, self.k, self.l = 1.0 / (N - 1), Ly / (N - 1), Lz / (N - 1)
        eye = sp.identity(N, format="csr")
        kr = lambda a, b, c: sp.kron(a, sp.kron(b, c, format="csr"), format="csr")
        # flattened index = x + N*y + N*N*z  ->  kron(z-factor, y-factor, x-factor)
        self.Dx = kr(eye, eye, _d1(N, self.h))
        self.Dy = kr(eye, _d1(N, self.k), eye)
        self.Dz = kr(_d1(N, self.l), eye, eye)
        self.Dxx = kr(eye, eye, _d2(N, self.h))
        self.Dyy = kr(eye, _d2(N, self.k), eye)
        self.Dzz = kr(_d2(N, self.l), eye, eye)
        # cross operators of the three edge groups of Eq. (5)
        self.Dxxyy = (self.Dxx @ self.Dyy).tocsr()
        self.Dxxy = (self.Dxx @ self.Dy).tocsr()
        self.Dxyy = (self.Dx @ self.Dyy).tocsr()
        self.Dxy = (self.Dx @ self.Dy).tocsr()
        self.Dyyzz = (self.Dyy @ self.Dzz).tocsr()
        self.Dyyz = (self.Dyy @ self.Dz).tocsr()
        self.Dyzz = (self.Dy @ self.Dzz).tocsr()
        self.Dyz = (self.Dy @ self.Dz).tocsr()
        self.Dzzxx = (self.Dzz @ self.Dxx).tocsr()
        self.Dzzx = (self.Dzz @ self.Dx).tocsr()
        self.Dzxx = (self.Dz @ self.Dxx).tocsr()
        self.Dzx = (self.Dz @ self.Dx).tocsr()
        interior = np.zeros((N, N, N), dtype=bool)
        interior[1:-1, 1:-1, 1:-1] = True
        self.interior = interior
        self.int_idx = np.flatnonzero(interior.ravel())
        self.bnd_idx = np.flatnonzero(~interior.ravel())
        self.x = np.linspace(0.0, 1.0, N)
        self.y = np.linspace(0.0, Ly, N)
        self.z = np.linspace(0.0, Lz, N)

    @classmethod
    def of(cls, prm):
        """The grid of a parameter set."""
        return cls(prm.N, prm.Ly, prm.Lz)

    def coords(self):
        z, y, x = np.meshgrid(self.z, self.y, self.x, indexing="ij")
        return x, y, z


# ------------------------------------------------------------ Eq. (5): the generic scalar scheme

def scalar_coefficients(g, dt, L, G, H, I, K, E, prev=None):
    """Coefficients of Eq. (5) for the generic transport equation (1).

    L, G, H, I, K, E are flattened level-n coefficient fields (L, G*, H*, I*, K*, E*); ``prev`` is
    a dict with the same keys at level n-1 (None at the first step, where delta_t^- = 0).
    Returns a dict with alpha, beta, gamma, M1..M4, R, p1, q1, r1 (Eq. 5 coefficient list) and the
    level-n fields themselves.
    """
    if prev is None:
        prev = dict(L=L, G=G, H=H, I=I, K=K, E=E)
    h2, k2, l2 = g.h ** 2, g.k ** 2, g.l ** 2

    def bracket(f, f_prev):
        # [1 + (dx^2 - G dx) h^2/12 + (dy^2 - H dy) k^2/12 + (dz^2 - I dz) l^2/12 + (dt/2) dt^-] f
        return (f
                + (g.Dxx @ f - G * (g.Dx @ f)) * (h2 / 12.0)
                + (g.Dyy @ f - H * (g.Dy @ f)) * (k2 / 12.0)
                + (g.Dzz @ f - I * (g.Dz @ f)) * (l2 / 12.0)
                + 0.5 * dt * (f - f_prev) / dt)

    c = {}
    c["alpha"] = (G * G - K - 2.0 * (g.Dx @ G)) * (h2 / 12.0) + 1.0
    c["gamma"] = (I * I - K - 2.0 * (g.Dz @ I)) * (l2 / 12.0) + 1.0
    c["beta"] = (H * H - K - 2.0 * (g.Dy @ H)) * (k2 / 12.0) + 1.0
    c["M1"] = bracket(G, prev["G"]) - (h2 / 12.0) * (G * K - 2.0 * (g.Dx @ K))
    c["M2"] = bracket(H, prev["H"]) - (k2 / 12.0) * (H * K - 2.0 * (g.Dy @ K))
    c["M3"] = bracket(I, prev["I"]) - (l2 / 12.0) * (I * K - 2.0 * (g.Dz @ K))
    c["M4"] = bracket(K, prev["K"])
    c["R"] = bracket(E, prev["E"])
    c["q1"] = -H * I + 2.0 / (k2 + l2) * (l2 * (g.Dz @ H) + k2 * (g.Dy @ I))
    c["p1"] = -G * H + 2.0 / (h2 + k2) * (k2 * (g.Dy @ G) + h2 * (g.Dx @ H))
    c["r1"] = -I * G + 2.0 / (l2 + h2) * (h2 * (g.Dx @ I) + l2 * (g.Dz @ G))
    c.update(L=L, G=G, H=H, I=I, K=K, E=E, L_prev=prev["L"])
    return c


def pseudo_time_mass(g, dt, c, kappa):
    """Reading R19: diagonal mass added to the level-(n+1) operator so that every grid mode of
    the frozen-coefficient pseudo-time update chi <- chi + dt A^-1 (R - B chi) is damped.

    The level-n operator B carries the compact correction (h^2/12)|G*|^2 delta^2 explicitly
    (inside alpha, beta, gamma); for the grid mode that alternates in all three directions the
    level-(n+1) operator reduces to 2 dt S with S = 1/h^2 + 1/k^2 + 1/l^2 (its compact mass
    cancels whatever the spacings), so that mode grows once |G*|^2 > 8 S (|G*|^2 h^2 > 24 on a
    cubic grid), and the mode alternating in one direction grows once dt |G*|^2 > 4 L.
    sigma = kappa * max(0, dt (|G*|^2/6 - S/3), dt |G*|^2/6 - 2 L/3) keeps both damped (S/3 =
    1/h^2 on a cubic grid). It is zero for well-resolved flows; A only sets the pseudo-time
    path, never the steady state.
    """
    G2 = c["G"] ** 2 + c["H"] ** 2 + c["I"] ** 2
    S = 1.0 / g.h ** 2 + 1.0 / g.k ** 2 + 1.0 / g.l ** 2
    sig = np.maximum(0.0, np.maximum(dt * (G2 / 6.0 - S / 3.0), dt * G2 / 6.0 - 2.0 * c["L"] / 3.0))
    return kappa * sig


def assemble_A(g, dt, c, a_limit=0.0, a_boost=0.0):
    """The level-(n+1) operator of Eq. (5): the bracket multiplying delta_t^+ chi, as a sparse matrix.

    Written term by term as printed in Eq. (5):
      L [ 1 - (dt/(2L) - k^2/12)(dy^2 - H dy) - (dt/(2L) - h^2/12)(dx^2 - G dx)
            - (dt/(2L) - l^2/12)(dz^2 - I dz)
            + dt/(2L) (K + dt^- L + h^2/(6dt) dx^2 L + k^2/(6dt) dy^2 L + l^2/(6dt) dz^2 L)
            + 1/(12 L) (-h^2 G dx L - l^2 I dz L - k^2 H dy L)
            + (k^2/(6L) dy L) dy + (h^2/(6L) dx L) dx + (l^2/(6L) dz L) dz ] .
    Its rows at interior nodes are the seven weights L1..L7 of Eq. (6).

    Reading R18: with a_limit > 0, the diagonal part M18 = L * (diagonal bracket terms other
    than K) is limited below by -a_limit * L, so that the extrapolated mass of the level-(n+1)
    operator stays positive when L drops fast between steps or varies strongly across a cell.
    A only sets the pseudo-time path; the steady state B chi = R does not involve it.
    """
    L, G, H, I, K = c["L"], c["G"], c["H"], c["I"], c["K"]
    h2, k2, l2 = g.h ** 2, g.k ** 2, g.l ** 2
    D = sp.diags
    dtL = dt / (2.0 * L)
    dL_t = (L - c["L_prev"]) / dt
    diag_terms = (dtL * (K + dL_t + h2 / (6 * dt) * (g.Dxx @ L) + k2 / (6 * dt) * (g.Dyy @ L)
                         + l2 / (6 * dt) * (g.Dzz @ L))
                  + 1.0 / (12.0 * L) * (-h2 * G * (g.Dx @ L) - l2 * I * (g.Dz @ L)
                                        - k2 * H * (g.Dy @ L)))
    if a_limit > 0.0:
        diag_terms = np.maximum(diag_terms - dtL * K, -a_limit) + dtL * K
    inner = (sp.identity(g.N ** 3, format="csr")
             - D(dtL - k2 / 12.0) @ (g.Dyy - D(H) @ g.Dy)
             - D(dtL - h2 / 12.0) @ (g.Dxx - D(G) @ g.Dx)
             - D(dtL - l2 / 12.0) @ (g.Dzz - D(I) @ g.Dz)
             + D(diag_terms)
             + D(k2 / (6.0 * L) * (g.Dy @ L)) @ g.Dy
             + D(h2 / (6.0 * L) * (g.Dx @ L)) @ g.Dx
             + D(l2 / (6.0 * L) * (g.Dz @ L)) @ g.Dz)
    A = D(L) @ inner
    if a_boost > 0.0:
        A = A + D(pseudo_time_mass(g, dt, c, a_boost))
    return A.tocsr()


def apply_B(g, c, chi):
    """The level-n operator of Eq. (5) applied to chi (19-point: centre, 6 faces, 12 edges):
      (-beta dy^2 - alpha dx^2 - gamma dz^2 + M2 dy + M4 + M1 dx + M3 dz) chi
      - (k^2+l^2)/12 (dy^2 dz^2 - I dy^2 dz - H dy dz^2 - q1 dy dz) chi
      - (h^2+k^2)/12 (dx^2 dy^2 - H dx^2 dy - G dx dy^2 - p1 dx dy) chi
      - (l^2+h^2)/12 (dz^2 dx^2 - G dz^2 dx - I dz dx^2 - r1 dz dx) chi .
    """
    G, H, I = c["G"], c["H"], c["I"]
    h2, k2, l2 = g.h ** 2, g.k ** 2, g.l ** 2
    out = (-c["beta"] * (g.Dyy @ chi) - c["alpha"] * (g.Dxx @ chi) - c["gamma"] * (g.Dzz @ chi)
           + c["M2"] * (g.Dy @ chi) + c["M4"] * chi + c["M1"] * (g.Dx @ chi)
           + c["M3"] * (g.Dz @ chi))
    out -= (k2 + l2) / 12.0 * (g.Dyyzz @ chi - I * (g.Dyyz @ chi) - H * (g.Dyzz @ chi)
                               - c["q1"] * (g.Dyz @ chi))
    out -= (h2 + k2) / 12.0 * (g.Dxxyy @ chi - H * (g.Dxxy @ chi) - G * (g.Dxyy @ chi)
                               - c["p1"] * (g.Dxy @ chi))
    out -= (l2 + h2) / 12.0 * (g.Dzzxx @ chi - G * (g.Dzzx @ chi) - I * (g.Dzxx @ chi)
                               - c["r1"] * (g.Dzx @ chi))
    return out


def solve_bicgstab(A, b, x0, tol, max_iter):
    """Unpreconditioned BiCGSTAB (van der Vorst 1992), the solver named in Sec. 2.2.

    Stops when ||r_k||_2 <= tol * ||r_0||_2 with r_0 = b - A x0. Returns (x, iterations, status)
    with status 0 = converged, 4 = iteration limit or breakdown.
    """
    x = x0.copy()
    r = b - A @ x
    r0n = math.sqrt(float(r @ r))
    if r0n == 0.0:
        return x, 0, 0
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, max_iter + 1):
        rho_new = float(rhat @ r)
        if rho_new == 0.0 or omega == 0.0:
            return x, it - 1, 4
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A @ p
        rv = float(rhat @ v)
        if rv == 0.0:
            return x, it - 1, 4
        alpha = rho_new / rv
        s = r - alpha * v
        t = A @ s
        tt = float(t @ t)
        omega = float(t @ s) / tt if tt > 0.0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        if math.sqrt(float(r @ r)) <= tol * r0n:
            return x, it, 0
    return x, max_iter, 4


def solve_bicgstab_l(A, b, x0, tol, max_iter, ell=2, trace=None):
    """BiCGSTAB(ell) (Sleijpen and Fokkema 1993): ell BiCG steps, then a minimal-residual update
    over the ell new residual directions (modified Gram-Schmidt), per cycle. A reading of the
    'hybrid' BiCGSTAB of Sec. 2.2 (a hybrid of BiCG and GMRES(ell)); ell = 1 is BiCGSTAB.

    The shadow residual is r_0 = b - A x0. Stops at the end of a cycle when ||r||_2 <= tol
    ||r_0||_2. Iterations are counted as ell per cycle (two operator applications each, the unit
    of solve_bicgstab). Returns (x, iterations, status), status 0 = converged, 4 = iteration
    limit or breakdown. ``trace``, when given, is called after every cycle with the residuals
    r_0..r_ell of the BiCG part (before the minimal-residual update) and the new residual.
    """
    x = x0.copy()
    r = [b - A @ x] + [None] * ell
    r0n = math.sqrt(float(r[0] @ r[0]))
    if r0n == 0.0:
        return x, 0, 0
    rt = r[0].copy()                       # shadow residual
    u = [np.zeros_like(b)] + [None] * ell
    rho0, alpha, omega = 1.0, 0.0, 1.0
    it = 0
    while it < max_iter:
        rho0 = -omega * rho0
        for j in range(ell):               # BiCG part
            rho1 = float(rt @ r[j])
            if rho0 == 0.0:
                return x, it, 4
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = A @ u[j]
            gam = float(rt @ u[j + 1])
            if gam == 0.0:
                return x, it, 4
            alpha = rho0 / gam
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = A @ r[j]
            x = x + alpha * u[0]
        # minimal-residual part: modified Gram-Schmidt on r_1..r_ell
        bicg = [v.copy() for v in r] if trace else None
        tau = np.zeros((ell + 1, ell + 1))
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1)             # gamma'
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = float(r[j] @ r[i]) / sigma[i]
                r[j] = r[j] - tau[i, j] * r[i]
            sigma[j] = float(r[j] @ r[j])
            if sigma[j] == 0.0:
                return x, it, 4
            gp[j] = float(r[0] @ r[j]) / sigma[j]
        g = np.zeros(ell + 1)              # gamma
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1)            # gamma''
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * r[0]
        r[0] = r[0] - gp[ell] * r[ell]
        u[0] = u[0] - g[ell] * u[ell]
        for j in range(1, ell):
            u[0] = u[0] - g[j] * u[j]
            x = x + gpp[j] * r[j]
            r[0] = r[0] - gp[j] * r[j]
        it += ell
        if trace:
            trace(bicg, r[0].copy())
        rn = math.sqrt(float(r[0] @ r[0]))
        if not math.isfinite(rn):
            return x, it, 4
        if rn <= tol * r0n:
            return x, it, 0
    return x, it, 4


def solve_system(g, dt, c, A, chi, tol, max_iter, direct=False, chi_wall_new=None,
                 precond=0, solver=0):
    """One implicit HOSC solve, Eq. (6): A chi^{n+1} = Q chi^n + dt R with Q = A - dt B.

    Unknowns are the interior nodes. Wall values of chi^{n+1} are ``chi_wall_new`` when given
    (a field whose wall nodes hold level-(n+1) values), else the level-n wall values (reading R6).
    With precond = 1 every row of the interior system and its right-hand side are divided by the
    row's diagonal entry before BiCGSTAB (Jacobi row scaling; the solution does not change).
    solver = 1 selects BiCGSTAB(2) (solve_bicgstab_l) instead of BiCGSTAB.
    Returns (chi_new, iterations, status).
    """
    chi_f = chi.ravel()
    b_full = A @ chi_f - dt * apply_B(g, c, chi_f) + dt * c["R"]
    ii, bb = g.int_idx, g.bnd_idx
    wall = chi_f if chi_wall_new is None else chi_wall_new.ravel()
    A_rows = A[ii]
    A_II = A_rows[:, ii].tocsr()
    A_IB = A_rows[:, bb]
    rhs = b_full[ii] - A_IB @ wall[bb]
    if precond:
        d = A_II.diagonal()
        d = np.where(d != 0.0, d, 1.0)
        A_II = (sp.diags(1.0 / d) @ A_II).tocsr()
        rhs = rhs / d
    if direct:
        import scipy.sparse.linalg as spla
        x, its, st = spla.spsolve(A_II.tocsc(), rhs), 0, 0
    elif solver == 1:
        x, its, st = solve_bicgstab_l(A_II, rhs, chi_f[ii], tol, max_iter, ell=2)
    else:
        x, its, st = solve_bicgstab(A_II, rhs, chi_f[ii], tol, max_iter)
    out = wall.copy()
    out[ii] = x
    return out.reshape(chi.shape), its, st


# ------------------------------------------------------- physics: viscosity, sources, boundaries

def grad_full(f, axis, dx):
    """Derivative of f along ``axis`` (0=z, 1=y, 2=x) at every node: central at nodes interior
    along that axis, second-order one-sided at the two walls (reading R7)."""
    f = np.moveaxis(f, axis, 0)
    d = np.empty_like(f)
    d[1:-1] = (f[2:] - f[:-2]) / (2.0 * dx)
    d[0] = (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * dx)
    d[-1] = (3.0 * f[-1] - 4.0 * f[-2] + f[-3]) / (2.0 * dx)
    return np.moveaxis(d, 0, axis)


def strain_gradients(u, v, w, h, k=None, l=None):
    """All nine velocity gradients at every node (keys 'ux', 'uy', ... ; reading R7); spacings
    h, k, l along x, y, z (k = l = h when not given)."""
    k = h if k is None else k
    l = h if l is None else l
    out = {}
    for name, f in (("u", u), ("v", v), ("w", w)):
        out[name + "x"] = grad_full(f, 2, h)
        out[name + "y"] = grad_full(f, 1, k)
        out[name + "z"] = grad_full(f, 0, l)
    return out


def second_invariant(gr):
    """I2 of Eq. (8): 2(u_x^2 + v_y^2 + w_z^2) + (u_z + w_x)^2 + (u_y + v_x)^2 + (v_z + w_y)^2."""
    return (2.0 * (gr["ux"] ** 2 + gr["vy"] ** 2 + gr["wz"] ** 2)
            + (gr["uz"] + gr["wx"]) ** 2 + (gr["uy"] + gr["vx"]) ** 2 + (gr["vz"] + gr["wy"]) ** 2)


def viscosity(u, v, w, prm):
    """Apparent viscosity eta = I2^((n-1)/2) (Eqs. 7-8) at every node, regularised (reading R1)."""
    gr = strain_gradients(u, v, w, *prm.spacings())
    I2 = second_invariant(gr)
    if prm.n == 1.0:
        eta = np.ones_like(I2)
    else:
        eta = (I2 + prm.I2_eps) ** (0.5 * (prm.n - 1.0))
        eta = edge_from_diagonal(eta)
    return eta, I2, gr


def edge_from_diagonal(f):
    """Reading R1b: on the 12 edges and 8 corners the one-sided strain rates of the two or three
    no-slip walls vanish identically, so I2 = 0 there whatever the flow. There the value is
    copied from the node one step inward along each wall normal the node lies on."""
    N = f.shape[0]
    out = f.copy()
    nb = lambda a: 1 if a == 0 else (N - 2 if a == N - 1 else a)
    wall = lambda a: a == 0 or a == N - 1
    for k in range(N):
        for j in range(N):
            for i in (range(N) if (wall(j) and wall(k)) else (0, N - 1)):
                if wall(i) + wall(j) + wall(k) >= 2:
                    out[k, j, i] = f[nb(k), nb(j), nb(i)]
    return out


def momentum_sources(u, v, w, th, p, eta, gr, prm):
    """E* of the three momentum equations at every node (Sec. 2.2 coefficient list, reading R2)."""
    h, k, l = prm.spacings()
    ex, ey, ez = grad_full(eta, 2, h), grad_full(eta, 1, k), grad_full(eta, 0, l)
    px, py, pz = grad_full(p, 2, h), grad_full(p, 1, k), grad_full(p, 0, l)
    exx, eyy, ezz = gr["ux"], gr["vy"], gr["wz"]
    exy = 0.5 * (gr["uy"] + gr["vx"])
    exz = 0.5 * (gr["uz"] + gr["wx"])
    eyz = 0.5 * (gr["vz"] + gr["wy"])
    Pr = prm.Pr
    Eu = -px / (Pr * eta) + (2.0 / eta) * (exx * ex + exy * ey + exz * ez)
    Ev = (-py / (Pr * eta) + (2.0 / eta) * (exy * ex + eyy * ey + eyz * ez)
          + prm.Ra * (th - prm.theta_ref) / eta)
    Ew = -pz / (Pr * eta) + (2.0 / eta) * (exz * ex + eyz * ey + ezz * ez)
    return Eu, Ev, Ew


def apply_theta_bc(th):
    """theta = 1 on x=0, theta = 0 on x=1 (whole faces); on the adiabatic y and z walls
    theta_b = (4 theta_1 - theta_2)/3 (reading R6/R7), y walls first, then z walls."""
    th = th.copy()
    th[:, :, 0] = 1.0
    th[:, :, -1] = 0.0
    th[1:-1, 0, 1:-1] = (4.0 * th[1:-1, 1, 1:-1] - th[1:-1, 2, 1:-1]) / 3.0
    th[1:-1, -1, 1:-1] = (4.0 * th[1:-1, -2, 1:-1] - th[1:-1, -3, 1:-1]) / 3.0
    th[0, :, 1:-1] = (4.0 * th[1, :, 1:-1] - th[2, :, 1:-1]) / 3.0
    th[-1, :, 1:-1] = (4.0 * th[-2, :, 1:-1] - th[-3, :, 1:-1]) / 3.0
    return th


def apply_pressure_bc(p):
    """Zero normal pressure gradient on every wall (Sec. 2.1), p_b = (4 p_1 - p_2)/3 (reading R5):
    x walls (interior y, z), then y walls (all x, interior z), then z walls (all x, y)."""
    p = p.copy()
    p[1:-1, 1:-1, 0] = (4.0 * p[1:-1, 1:-1, 1] - p[1:-1, 1:-1, 2]) / 3.0
    p[1:-1, 1:-1, -1] = (4.0 * p[1:-1, 1:-1, -2] - p[1:-1, 1:-1, -3]) / 3.0
    p[1:-1, 0, :] = (4.0 * p[1:-1, 1, :] - p[1:-1, 2, :]) / 3.0
    p[1:-1, -1, :] = (4.0 * p[1:-1, -2, :] - p[1:-1, -3, :]) / 3.0
    p[0, :, :] = (4.0 * p[1, :, :] - p[2, :, :]) / 3.0
    p[-1, :, :] = (4.0 * p[-2, :, :] - p[-3, :, :]) / 3.0
    return p


def divergence(u, v, w, h, k=None, l=None):
    """Central div V at interior nodes (zero elsewhere); spacings h, k, l along x, y, z (k = l =
    h when not given)."""
    k = h if k is None else k
    l = h if l is None else l
    D = np.zeros_like(u)
    D[1:-1, 1:-1, 1:-1] = ((u[1:-1, 1:-1, 2:] - u[1:-1, 1:-1, :-2]) / (2.0 * h)
                           + (v[1:-1, 2:, 1:-1] - v[1:-1, :-2, 1:-1]) / (2.0 * k)
                           + (w[2:, 1:-1, 1:-1] - w[:-2, 1:-1, 1:-1]) / (2.0 * l))
    return D


# --------------------------------------------------------------------------------- time step

def initial_state(prm):
    """Fluid at rest: zero velocity, constant (zero) pressure (Sec. 2.2 'constant initial
    pressure'), theta = theta_init inside (reading R12, default 1/2) with the wall conditions."""
    N = prm.N
    z = np.zeros((N, N, N))
    return dict(u=z.copy(), v=z.copy(), w=z.copy(), th=apply_theta_bc(z + prm.theta_init),
                p=z.copy(), prev=None, steps=0)


def level_coefficients(state, prm):
    """Level-n coefficient fields of the four systems (Sec. 2.2 coefficient list)."""
    u, v, w, th, p = (state[k] for k in ("u", "v", "w", "th", "p"))
    eta, I2, gr = viscosity(u, v, w, prm)
    Eu, Ev, Ew = momentum_sources(u, v, w, th, p, eta, gr, prm)
    L = 1.0 / (prm.Pr * eta)
    return dict(eta=eta, L=L, u=u, v=v, w=w, Eu=Eu, Ev=Ev, Ew=Ew)


def _system_coefficients(g, prm, lev, prev):
    f = lambda a: a.ravel()
    zero = np.zeros(g.N ** 3)
    one = np.ones(g.N ** 3)
    mom = dict(L=f(lev["L"]), G=f(lev["u"] * lev["L"]), H=f(lev["v"] * lev["L"]),
               I=f(lev["w"] * lev["L"]), K=zero)
    ene = dict(L=one, G=f(lev["u"]), H=f(lev["v"]), I=f(lev["w"]), K=zero, E=zero)
    if prev is None:
        pm = pe = None
        pE = {}
    else:
        pm = dict(L=f(prev["L"]), G=f(prev["u"] * prev["L"]), H=f(prev["v"] * prev["L"]),
                  I=f(prev["w"] * prev["L"]), K=zero)
        pe = dict(L=one, G=f(prev["u"]), H=f(prev["v"]), I=f(prev["w"]), K=zero, E=zero)
        pE = dict(u=f(prev["Eu"]), v=f(prev["Ev"]), w=f(prev["Ew"]))
    out = {}
    for name, key in (("u", "Eu"), ("v", "Ev"), ("w", "Ew")):
        m = dict(mom, E=f(lev[key]))
        pmm = None if pm is None else dict(pm, E=pE[name])
        out[name] = scalar_coefficients(g, prm.dt, prev=pmm, **m)
    out["th"] = scalar_coefficients(g, prm.dt, prev=pe, **ene)
    return out


def relaxation(prm, eta):
    """The relaxation of the pressure correction p <- p - lam_c div V (Sec. 2.2): the scalar lam,
    or (reading R25, lam_mode = 1) lam_c = min(lam eta, 0.9 h^2/dt) node by node, so that the
    correction follows the viscous time scale of the local pressure modes. The fixed point
    div V = 0 does not depend on it."""
    if not prm.lam_mode:
        return prm.lam
    h = min(prm.spacings())
    return np.minimum(prm.lam * eta, 0.9 * h * h / prm.dt)


def step(state, prm, g=None, direct=False):
    """Advance one pseudo-time step n -> n+1 (Sec. 2.2 solution procedure). Returns (state, info).

    1. eta, L and E* at level n;  2. four HOSC solves (u, v, w, theta) with level-n coefficients;
    3. theta wall update;  4. div V^{n+1}, artificial-compressibility pressure correction;
    5. steady-state change r_n = max over u, v, w, theta of |chi^{n+1} - chi^n|.
    """
    g = g or Grid.of(prm)
    lev = level_coefficients(state, prm)
    coefs = _system_coefficients(g, prm, lev, state["prev"] if prm.use_history else None)
    A_m = assemble_A(g, prm.dt, coefs["u"], prm.a_limit, prm.a_boost)
    A_e = assemble_A(g, prm.dt, coefs["th"], prm.a_limit, prm.a_boost)
    new, iters, status = {}, {}, 0
    for name in ("u", "v", "w", "th"):
        A = A_e if name == "th" else A_m
        new[name], iters[name], st = solve_system(g, prm.dt, coefs[name], A, state[name],
                                                  prm.tol_lin, prm.max_lin_iter, direct=direct,
                                                  precond=prm.precond, solver=prm.solver)
        status = status or st
    new["th"] = apply_theta_bc(new["th"])
    sp3 = (g.h, g.k, g.l)
    D = divergence(new["u"], new["v"], new["w"], *sp3)
    d_max = float(np.max(np.abs(D)))
    p = state["p"].copy()
    lam = relaxation(prm, lev["eta"])
    if d_max > prm.tol_div:
        p = apply_pressure_bc(p - lam * D)
    # Inner pressure iterations (Sec. 2.2: the divergence is checked after the momentum equations
    # are solved, and while it exceeds the tolerance the pressure of the previous pressure
    # iteration is corrected; reading: the momentum systems are then solved again). Each pass
    # recomputes E* from the level-n velocities and viscosity with the corrected pressure and the
    # new temperature, solves u, v, w again from level n with the level-n operator, and corrects
    # the pressure; theta is not solved again (its system does not involve the pressure).
    inner = 0
    while prm.inner_max and d_max > prm.tol_div and inner < prm.inner_max:
        inner += 1
        lev = level_coefficients(dict(state, th=new["th"], p=p), prm)
        coefs = _system_coefficients(g, prm, lev, state["prev"] if prm.use_history else None)
        for name in ("u", "v", "w"):
            new[name], iters[name], st = solve_system(g, prm.dt, coefs[name], A_m, state[name],
                                                      prm.tol_lin, prm.max_lin_iter,
                                                      direct=direct, precond=prm.precond,
                                                      solver=prm.solver)
            status = status or st
        D = divergence(new["u"], new["v"], new["w"], *sp3)
        d_max = float(np.max(np.abs(D)))
        if d_max > prm.tol_div:
            p = apply_pressure_bc(p - lam * D)
    res = max(float(np.max(np.abs(new[k] - state[k]))) for k in ("u", "v", "w", "th"))
    out = dict(u=new["u"], v=new["v"], w=new["w"], th=new["th"], p=p,
               prev=dict(L=lev["L"], u=state["u"], v=state["v"], w=state["w"], Eu=lev["Eu"],
                         Ev=lev["Ev"], Ew=lev["Ew"]),
               steps=state["steps"] + 1)
    if not all(np.all(np.isfinite(out[k])) for k in ("u", "v", "w", "th", "p")):
        status = 5
    info = dict(res=res, div_max=d_max, iters=iters, status=status, inner=inner)
    return out, info


def solve_steady(prm, max_steps, tol_steady=1e-6, state=None, g=None, callback=None,
                 div_stop=None):
    """March to steady state: stop when r_n < tol_steady and max|div V| < div_stop
    (default tol_div)."""
    g = g or Grid.of(prm)
    state = state or initial_state(prm)
    div_stop = prm.tol_div if div_stop is None else div_stop
    info = None
    for _ in range(max_steps):
        state, info = step(state, prm, g)
        if callback:
            callback(state, info)
        if info["status"]:
            break
        if info["res"] < tol_steady and info["div_max"] < div_stop:
            break
    return state, info


def steady_certificate(state, prm, g=None):
    """Steady residuals of a field set: max over the four systems of |B chi - R| at interior nodes
    (the dt-free fixed-point equation of Eq. 5) and max|div V|."""
    g = g or Grid.of(prm)
    st = dict(state, prev=None)
    lev = level_coefficients(st, prm)
    coefs = _system_coefficients(g, prm, lev, None)
    worst = 0.0
    for name in ("u", "v", "w", "th"):
        r = apply_B(g, coefs[name], state[name].ravel()) - coefs[name]["R"]
        worst = max(worst, float(np.max(np.abs(r[g.int_idx]))))
    D = divergence(state["u"], state["v"], state["w"], g.h, g.k, g.l)
    return worst, float(np.max(np.abs(D)))


# --------------------------------------------------------------------------------- diagnostics

def simpson_weights(N, h):
    """Composite Simpson weights on N nodes (N odd); trapezoid weights when N is even."""
    wts = np.empty(N)
    if N % 2 == 1:
        wts[:] = 2.0
        wts[1:-1:2] = 4.0
        wts[0] = wts[-1] = 1.0
        return wts * h / 3.0
    wts[:] = 1.0
    wts[0] = wts[-1] = 0.5
    return wts * h


def diagnostics(state, prm):
    """Nusselt numbers (Sec. 4.2) and entropy generation / Bejan number (Sec. 4.3).

    Returns a dict: Nu_hot_local[z, y], Nu_avg_z[z], Nu_hot_max, Nu_hot_mean, Nu_cold_mean,
    E_HT, E_FF, E_local (fields), E_total, E_HT_total, E_FF_total, Be, Be_local. On a box
    1 x Ly x Lz the wall averages are over the wall (Nu_avg_z: mean over y; Nu_mean: over y and
    z) and the entropy totals are integrals over the box volume.
    """
    N = prm.N
    h, k, l = prm.spacings()
    th = state["th"]
    # fourth-order one-sided d theta/dx at x = 0 and x = 1 (reading R10)
    dth0 = (-25.0 * th[:, :, 0] + 48.0 * th[:, :, 1] - 36.0 * th[:, :, 2] + 16.0 * th[:, :, 3]
            - 3.0 * th[:, :, 4]) / (12.0 * h)
    dth1 = (25.0 * th[:, :, -1] - 48.0 * th[:, :, -2] + 36.0 * th[:, :, -3]
            - 16.0 * th[:, :, -4] + 3.0 * th[:, :, -5]) / (12.0 * h)
    nu_hot = -dth0
    nu_cold = -dth1
    wx, wy, wz = simpson_weights(N, h), simpson_weights(N, k), simpson_weights(N, l)
    area = prm.Ly * prm.Lz
    nu_avg_z = nu_hot @ wy / prm.Ly
    out = dict(Nu_hot_local=nu_hot, Nu_avg_z=nu_avg_z, Nu_hot_max=float(np.max(nu_avg_z)),
               Nu_hot_mean=float(wz @ nu_hot @ wy) / area,
               Nu_cold_mean=float(wz @ nu_cold @ wy) / area)
    eta, I2, _ = viscosity(state["u"], state["v"], state["w"], prm)
    E_HT = grad_full(th, 2, h) ** 2 + grad_full(th, 1, k) ** 2 + grad_full(th, 0, l) ** 2
    E_FF = prm.phi * eta * I2
    E_loc = E_HT + E_FF
    vol = lambda f: float(np.einsum("zyx,z,y,x->", f, wz, wy, wx))
    t_ht, t_ff = vol(E_HT), vol(E_FF)
    be_loc = np.where(E_loc > 0.0, E_HT / np.where(E_loc > 0.0, E_loc, 1.0), 1.0)
    out.update(E_HT=E_HT, E_FF=E_FF, E_local=E_loc, E_HT_total=t_ht, E_FF_total=t_ff,
               E_total=t_ht + t_ff, Be=t_ht / (t_ht + t_ff), Be_local=be_loc)
    return out
