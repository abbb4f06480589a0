"""GPU parity at the sizes of the workloads the library is run and measured at, through the C ABI,
against the FP64 oracle.

* the benched single cavity (101^3, n = 0.75, Ra = 1e5, Pr = 1): one step from a seeded developed
  state at the launch shape the autotuner picks, all-FP64 (fields 1e-10 relative) and mixed
  precision (each field's change within 1e-3 of the oracle's change, and the FP32 solution's
  residual in the oracle's system, see MIXED_TOL);
* the power-law 41^3 cavities (Ra = 1e4, n = 0.75 and 1.25): a short FP64 trajectory at the
  workload's pseudo-time step (1e-10), and one mixed step (as above);
* the scheme exactly as printed (no M18 limiter, no pseudo-time mass): an FP64 trajectory from
  rest (1e-10) and a mixed one (1e-5 of the fields).

Tolerances: 1e-10 relative is the all-FP64 target; the mixed path solves each level-(n+1) system
in FP32 to a relative residual of 3e-6 (see MIXED_TOL for what that bounds).
"""

import numpy as np
import pytest

from oracle import hosc_oracle as O

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2411_06563_gb300.hosc")
from paper_2411_06563_gb300 import inputs  # noqa: E402

FIELDS = (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA),
          ("p", H.HOSC_P))


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _oracle_params(p):
    return O.Params(N=p.N, Ra=p.Ra, Pr=p.Pr, n=p.n, dt=p.dt, lam=p.lambda_,
                    theta_ref=p.theta_ref, I2_eps=p.I2_eps, phi=p.phi, tol_div=p.tol_div,
                    tol_lin=p.tol_lin, max_lin_iter=p.max_lin_iter, theta_init=p.theta_init,
                    a_limit=p.a_limit, a_boost=p.a_boost, use_history=p.use_history,
                    precond=p.precond, inner_max=p.inner_max, Ly=p.Ly or 1.0, Lz=p.Lz or 1.0,
                    solver=p.solver, lam_mode=p.lambda_mode)


def _params(N, Ra, n, dt, lam, precision, tol_lin, **kw):
    p = H.hosc_default_params(N, Ra, 1.0, n)
    p.dt, p.lambda_, p.tol_lin, p.max_lin_iter = dt, lam, tol_lin, 4000
    p.precision = precision
    p.auto_defect = 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _load(cav, st):
    for name, which in FIELDS:
        cav.set(which, st[name])


def _check_change(got, st0, ref, name, tol):
    """The GPU's change of a field over the step against the oracle's, relative to the size of
    the oracle's change."""
    inc = ref - st0
    scale = max(float(np.max(np.abs(inc))), 1e-12)
    err = float(np.max(np.abs((got - st0) - inc)))
    assert err <= tol * scale, (name, err / scale)


# --------------------------------------------------------------- the benched 101^3 cavity

N101, RA101, N_IDX101, DT101, LAM101 = 101, 1e5, 0.75, 2e-5, 0.3


@pytest.fixture(scope="module")
def step101():
    """The oracle's step from the seeded 101^3 state (about 4 s on the host, plus the sparse
    operators)."""
    st = dict(inputs.cavity_state(N101, RA101, seed=1010), prev=None, steps=0)
    p = _params(N101, RA101, N_IDX101, DT101, LAM101, H.HOSC_FP64, 1e-12)
    op = _oracle_params(p)
    new, info = O.step(st, op, O.Grid.of(op))
    assert info["status"] == 0
    return st, new, info


# Mixed precision, one step against the FP64 oracle's step. The level-(n+1) systems are solved in
# FP32 until the relative residual is 3e-6, so the increment carries a relative error of up to
# kappa(A) * 3e-6: about 3e-4 of the largest change at 101^3 (kappa ~ 100 for the advective
# momentum operators at this cell Reynolds number), 1e-4 at 41^3. The change is checked to 1e-3 of
# its size, and, with FP64 sweeps (phase 1, the right-hand side evaluated in double), the FP32
# solution is checked directly against the oracle's system: ||A x_gpu - b||_2 <= 3e-5 ||b||_2 for
# each of the four systems (the 3e-6 stopping test plus the float rounding of the operator and
# of the vectors). With FP32 sweeps (phase 0) the right-hand side is a float evaluation of the
# oracle's, so only the change is compared.
MIXED_TOL = {0: 1e-3, 1: 1e-3}
RESID_TOL = 3e-5


def _increment_residuals(st0, got, op):
    """||A x - b||_2 / ||b||_2 of the GPU's increments x in the oracle's increment systems
    A (chi^{n+1} - chi^n) = dt (R - B chi^n) at interior nodes (u, v, w, theta)."""
    g = O.Grid.of(op)
    ii = g.int_idx
    lev = O.level_coefficients(dict(st0, prev=None), op)
    coefs = O._system_coefficients(g, op, lev, None)
    A_m = O.assemble_A(g, op.dt, coefs["u"], op.a_limit, op.a_boost)[ii][:, ii]
    A_e = O.assemble_A(g, op.dt, coefs["th"], op.a_limit, op.a_boost)[ii][:, ii]
    out = {}
    for name in ("u", "v", "w", "th"):
        c = coefs[name]
        b = op.dt * (c["R"] - O.apply_B(g, c, st0[name].ravel()))[ii]
        x = (got[name] - st0[name]).ravel()[ii]
        A = A_e if name == "th" else A_m
        out[name] = float(np.linalg.norm(A @ x - b) / max(np.linalg.norm(b), 1e-300))
    return out


@pytest.mark.parametrize("precision,phase,shape", [(H.HOSC_FP64, 0, None),
                                                   (H.HOSC_MIXED, 0, "autotuned"),
                                                   (H.HOSC_MIXED, 1, "autotuned"),
                                                   (H.HOSC_MIXED, 1, (2, 33, 6, 1)),
                                                   (H.HOSC_MIXED, 0, (2, 17, 4, 3))])
def test_benched_cavity_101_one_step(step101, precision, phase, shape):
    """One step of the benched cavity from a seeded developed state against the oracle's step:
    FP64 fields within 1e-10; mixed precision at the autotuner's launch shape for this grid (the
    one the benchmark times) and with the bulk-copy stencil kernels forced (p/v alone, 2 rows x
    33 planes per block in a ring of six stages; both, 2 rows x 17 planes in a ring of four),
    within the FP32 solve's tolerance and, with FP64 sweeps, by residual in the oracle's
    system."""
    st0, ref, oinfo = step101
    tol_lin = 1e-12 if precision == H.HOSC_FP64 else 1e-10
    p = _params(N101, RA101, N_IDX101, DT101, LAM101, precision, tol_lin)
    with H.Cavity(p) as cav:
        _load(cav, st0)
        if precision == H.HOSC_MIXED:
            cav.step(1)
            if shape == "autotuned":
                rc, kb, kz, _ = H.hosc_autotune(cav.h, 3)
                assert rc == 0 and kb > 0 and kz > 0
            else:
                assert H.hosc_set_tma_tiles(cav.h, *shape) == 0
                assert H.hosc_get_tma_tiles(cav.h) == (0,) + tuple(shape)
            _load(cav, st0)
            cav.clear_history()
            assert H.hosc_set_phase(cav.h, phase) == 0
        info = cav.step(1)
        assert info["call_status"] == 0, info
        gotf = {}
        for name, which in FIELDS:
            got = gotf[name] = cav.get(which)
            if precision == H.HOSC_FP64:
                assert _rel(got, ref[name]) <= 1e-10, name
            else:
                _check_change(got, st0[name], ref[name], name, MIXED_TOL[phase])
        if precision == H.HOSC_MIXED and phase == 1:
            res = _increment_residuals(st0, gotf, _oracle_params(p))
            assert max(res.values()) <= RESID_TOL, res
        if precision == H.HOSC_FP64:
            assert abs(info["div_max"] - oinfo["div_max"]) <= 1e-9 * oinfo["div_max"]
            assert abs(info["res"] - oinfo["res"]) <= 1e-9 * oinfo["res"]


# --------------------------------------------------------------- the power-law 41^3 cavities

def _dt41(n):
    # the pseudo-time step of the steady-solve rule for these cavities (Ra = 1e4, Pr = 1)
    return H.hosc_steady_params(41, 1e4, 1.0, n).dt


@pytest.mark.parametrize("n", [0.75, 1.25])
def test_power_law_41_fp64_trajectory(n):
    """Five FP64 steps from a seeded developed state with history terms at the workload's
    pseudo-time step: every field after every step within 1e-10 of the oracle's."""
    N, Ra = 41, 1e4
    dt = _dt41(n)
    p = _params(N, Ra, n, dt, min(0.9 / (N - 1) ** 2 / dt, 0.5), H.HOSC_FP64, 1e-12,
                use_history=1)
    op = _oracle_params(p)
    g = O.Grid.of(op)
    st = dict(inputs.cavity_state(N, Ra, seed=41 + int(100 * n)), prev=None, steps=0)
    with H.Cavity(p) as cav:
        _load(cav, st)
        for _ in range(5):
            info = cav.step(1)
            st, oinfo = O.step(st, op, g)
            assert info["call_status"] == 0 and oinfo["status"] == 0
            for name, which in FIELDS:
                assert _rel(cav.get(which), st[name]) <= 1e-10, name
            for s_, name in enumerate(("u", "v", "w", "th")):
                it_o = oinfo["iters"][name]
                assert abs(info["last_iters"][s_] - it_o) <= 2 + it_o // 10


@pytest.mark.parametrize("n", [0.75, 1.25])
def test_power_law_41_mixed_step(n):
    N, Ra = 41, 1e4
    dt = _dt41(n)
    lam = min(0.9 / (N - 1) ** 2 / dt, 0.5)
    st0 = dict(inputs.cavity_state(N, Ra, seed=4100 + int(100 * n)), prev=None, steps=0)
    op = _oracle_params(_params(N, Ra, n, dt, lam, H.HOSC_FP64, 1e-12))
    ref, _ = O.step(st0, op, O.Grid.of(op))
    for phase in (0, 1):
        p = _params(N, Ra, n, dt, lam, H.HOSC_MIXED, 1e-10)
        with H.Cavity(p) as cav:
            _load(cav, st0)
            assert H.hosc_set_phase(cav.h, phase) == 0
            info = cav.step(1)
            assert info["call_status"] == 0
            gotf = {}
            for name, which in FIELDS:
                gotf[name] = cav.get(which)
                _check_change(gotf[name], st0[name], ref[name], name, MIXED_TOL[phase])
            if phase == 1:
                res = _increment_residuals(st0, gotf, op)
                assert max(res.values()) <= RESID_TOL, res


# --------------------------------------------------------------- the scheme as printed

def test_printed_scheme_without_limiter_or_mass():
    """a_limit = a_boost = 0 (readings R18 and R19 off: the level-(n+1) operator exactly as
    Eq. (5) prints it): twenty FP64 steps from rest of a 21^3 power-law cavity at a pseudo-time
    step inside the printed scheme's stability bound agree with the oracle's to 1e-10; the mixed
    path (FP64 sweeps, the printed operator solved in FP32) stays within 1e-5 of the fields."""
    N, Ra, n, dt = 21, 1e3, 0.75, 0.002
    lam = 0.5
    out = {}
    for precision in (H.HOSC_FP64, H.HOSC_MIXED):
        p = _params(N, Ra, n, dt, lam, precision, 1e-12 if precision == H.HOSC_FP64 else 1e-10,
                    a_limit=0.0, a_boost=0.0, use_history=1)
        op = _oracle_params(p)
        assert op.a_limit == 0.0 and op.a_boost == 0.0
        g = O.Grid.of(op)
        st = O.initial_state(op)
        with H.Cavity(p) as cav:
            if precision == H.HOSC_MIXED:
                assert H.hosc_set_phase(cav.h, 1) == 0   # FP64 sweeps, FP32 solve
            for k in range(20):
                info = cav.step(1)
                st, oinfo = O.step(st, op, g)
                assert info["call_status"] == 0 and oinfo["status"] == 0
                if precision == H.HOSC_FP64 or k == 19:
                    for name, which in FIELDS:
                        got = cav.get(which)
                        if precision == H.HOSC_FP64:
                            assert _rel(got, st[name]) <= 1e-10, (k, name)
                        else:
                            assert np.max(np.abs(got - st[name])) <= 1e-5 * max(
                                1.0, np.max(np.abs(st[name]))), (k, name)
        out[precision] = st


# --------------------------------------------------------------- the Newtonian 21^3 cavity

def _c1_params(precision):
    """The Newtonian 21^3 configuration (n = 1, Pr = 1, Ra = 1e3) with the library's pseudo-time
    step and relaxation for steady solves, stopped at max|chi^{n+1} - chi^n|/dt < 1e-6 and
    max|div V| < 1e-6 (div_steady; the pressure is corrected while max|div V| > tol_div)."""
    p = H.hosc_steady_params(21, 1e3, 1.0, 1.0)
    p.precision = precision
    p.tol_lin = 1e-12 if precision == H.HOSC_FP64 else 1e-10
    p.max_lin_iter = 4000
    return p


@pytest.fixture(scope="module")
def c1_march():
    """The GPU's FP64 steady solve of the configuration from rest, and the oracle marched the
    same number of steps from rest with the same parameters."""
    p = _c1_params(H.HOSC_FP64)
    with H.Cavity(p) as cav:
        info = cav.solve_steady(20000)
        assert info["call_status"] == 0, info
        gpu = {name: cav.get(which) for name, which in FIELDS}
        diag = cav.diagnostics()
    op = _oracle_params(p)
    g = O.Grid.of(op)
    st = O.initial_state(op)
    oinfo = None
    for _ in range(info["steps"]):
        prev_info = oinfo
        st, oinfo = O.step(st, op, g)
        assert oinfo["status"] == 0
    return p, info, gpu, diag, st, oinfo, prev_info


def test_newtonian_21_steady_state_fp64(c1_march):
    """The all-FP64 GPU steady solve stops at the step where the oracle's march meets the same
    stop rule (and not before), and its fields, step change, divergence and Nusselt numbers
    there agree with the oracle's to 1e-10 relative."""
    p, info, gpu, diag, st, oinfo, prev = c1_march
    stop = p.tol_steady * p.dt
    assert p.div_steady == 1e-6
    assert oinfo["res"] < stop and oinfo["div_max"] < p.div_steady
    assert not (prev["res"] < stop and prev["div_max"] < p.div_steady)
    for name, _ in FIELDS:
        assert _rel(gpu[name], st[name]) <= 1e-10, name
    # max|div V| is a difference of O(1) velocities over 2h: it agrees to rounding of that scale
    h = 1.0 / (p.N - 1)
    vmax = max(np.max(np.abs(st[k])) for k in ("u", "v", "w"))
    assert abs(info["div_max"] - oinfo["div_max"]) <= 1e-12 * vmax / h
    od = O.diagnostics(st, _oracle_params(p))
    for k_gpu, k_ora in (("Nu_hot_max", "Nu_hot_max"), ("Nu_hot_mean", "Nu_hot_mean"),
                         ("Nu_cold_mean", "Nu_cold_mean"), ("E_total", "E_total"),
                         ("Be", "Be")):
        assert diag[k_gpu] == pytest.approx(od[k_ora], rel=1e-10), k_gpu
    # a steady state of Eq. (5): the dt-free residual B chi - R is small on the GPU's fields
    cert, dmax = O.steady_certificate(gpu, _oracle_params(p))
    assert dmax < p.div_steady and cert < 1e-3


@pytest.mark.parametrize("mode", [H.HOSC_POOL_GRAPH, H.HOSC_POOL_STREAMS])
def test_newtonian_21_pool_members_against_the_oracle(c1_march, mode):
    """The same configuration solved as pool members beside two other cavities: the FP64
    member's steady fields equal the oracle's at its stop to 1e-10; the mixed-precision member
    (FP32 sweeps and solves, FP64 defect sweeps once the step change stalls) reaches the
    oracle's steady state within 1e-5 of the fields and 1e-4 of the mean Nusselt number."""
    from paper_2411_06563_gb300 import serve
    p64, _, _, _, st, _, _ = c1_march
    od = O.diagnostics(st, _oracle_params(p64))
    with serve.Pool(4 << 30, steps_per_round=16, mode=mode, autotune=False) as pool:
        slots = {}
        for prec in (H.HOSC_FP64, H.HOSC_MIXED):
            slots[prec] = pool.admit(_c1_params(prec), 40000)
        for N, Ra, n in ((17, 3e3, 0.8), (25, 1e3, 1.2)):
            pool.admit(H.hosc_steady_params(N, Ra, 1.0, n), 3000)
        done = set()
        while not set(slots.values()) <= done:
            done |= set(pool.run(64))
        res = {prec: pool.result(s, FIELDS) for prec, s in slots.items()}
    r64 = res[H.HOSC_FP64]
    assert r64["status"] == H.HOSC_OK
    for name, _ in FIELDS:
        assert _rel(r64[name], st[name]) <= 1e-10, name
    rmx = res[H.HOSC_MIXED]
    assert rmx["status"] == H.HOSC_OK
    for name, _ in FIELDS:
        if name == "p":
            continue
        assert np.max(np.abs(rmx[name] - st[name])) <= 1e-5, name
    assert rmx["diag"]["Nu_hot_mean"] == pytest.approx(od["Nu_hot_mean"], rel=1e-4)
    assert rmx["diag"]["Nu_hot_max"] == pytest.approx(od["Nu_hot_max"], rel=1e-4)


# --------------------------------------------------------------- viscosity-scaled relaxation

@pytest.mark.parametrize("n", [0.75, 1.25])
def test_viscosity_scaled_relaxation_trajectory(n):
    """lambda_mode = 1 (reading R25: the pressure correction relaxed by lambda * eta node by
    node, at most 0.9 h^2/dt): six FP64 steps of a seeded 17^3 power-law state agree with the
    oracle's to 1e-10 (the cap is reached at some nodes and not at others), and a mixed step's
    change with FP64 sweeps within 2e-5."""
    N, Ra = 17, 1e4
    h = 1.0 / (N - 1)
    dt = 2e-4
    lam = 0.6 * 0.9 * h * h / dt
    st0 = dict(inputs.cavity_state(N, Ra, seed=1700 + int(100 * n)), prev=None, steps=0)
    p = _params(N, Ra, n, dt, lam, H.HOSC_FP64, 1e-12, lambda_mode=1, use_history=0)
    op = _oracle_params(p)
    assert op.lam_mode == 1
    g = O.Grid.of(op)
    eta, _, _ = O.viscosity(st0["u"], st0["v"], st0["w"], op)
    relax = O.relaxation(op, eta)
    assert np.any(relax < 0.9 * h * h / dt) and np.any(relax == 0.9 * h * h / dt)
    st = st0
    with H.Cavity(p) as cav:
        _load(cav, st)
        for _ in range(6):
            info = cav.step(1)
            st, oinfo = O.step(st, op, g)
            assert info["call_status"] == 0 and oinfo["status"] == 0
            for name, which in FIELDS:
                assert _rel(cav.get(which), st[name]) <= 1e-10, name
    ref, _ = O.step(st0, op, g)
    pm = _params(N, Ra, n, dt, lam, H.HOSC_MIXED, 1e-10, lambda_mode=1, use_history=0)
    with H.Cavity(pm) as cav:
        _load(cav, st0)
        assert H.hosc_set_phase(cav.h, 1) == 0
        assert cav.step(1)["call_status"] == 0
        gotf = {}
        for name, which in FIELDS:
            gotf[name] = cav.get(which)
            _check_change(gotf[name], st0[name], ref[name], name, MIXED_TOL[1])
        res = _increment_residuals(st0, gotf, op)
        assert max(res.values()) <= RESID_TOL, res
