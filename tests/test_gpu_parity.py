"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element, on
seeded synthetic states. One row of the hot path per check:

  S1 viscosity eta, L      S2 momentum sources E*      S3 right-hand sides dt (R - B chi^n)
  S4/S5 the level-(n+1) operator and BiCGSTAB (GPU increment vs oracle direct solve; oracle
        operator applied to the GPU increment reproduces the GPU right-hand side)
  S6-S8 one full step (u, v, w, theta, p), multi-step trajectories, diagnostics.

Tolerances (FP64 both sides): relative to the largest magnitude of the compared quantity,
1e-13 for eta and L, 1e-12 for E* (one division and a few products), 1e-11 for the right-hand
sides (19-point sums of O(1/h^4)-weighted terms), 1e-9 for the BiCGSTAB increment solved to
1e-13 against a direct solve, and 1e-10 for the fields after a step (the all-FP64 target).
"""

import numpy as np
import pytest

from oracle import hosc_oracle as O

pytestmark = pytest.mark.gpu

hosc = pytest.importorskip("paper_2411_06563_gb300.hosc")
from paper_2411_06563_gb300 import inputs  # noqa: E402

H = hosc


def _rel(a, b):
    scale = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / scale)


def _params(N, Ra, n, dt=0.01, Pr=1.0, tol_lin=1e-13, **kw):
    p = H.hosc_default_params(N, Ra, Pr, n)
    p.dt = dt
    p.lambda_ = 0.25 / (N - 1) ** 2 / dt
    p.tol_lin = tol_lin
    p.max_lin_iter = 3000
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _oracle_params(p):
    return O.Params(N=p.N, Ra=p.Ra, Pr=p.Pr, n=p.n, dt=p.dt, lam=p.lambda_,
                    theta_ref=p.theta_ref, I2_eps=p.I2_eps, phi=p.phi, tol_div=p.tol_div,
                    tol_lin=p.tol_lin, max_lin_iter=p.max_lin_iter, theta_init=p.theta_init,
                    a_limit=p.a_limit, a_boost=p.a_boost, use_history=p.use_history,
                    precond=p.precond, inner_max=p.inner_max, Ly=p.Ly or 1.0, Lz=p.Lz or 1.0,
                    solver=p.solver, lam_mode=p.lambda_mode)


def _setup(N, Ra, n, seed, history, **kw):
    p = _params(N, Ra, n, **kw)
    op = _oracle_params(p)
    st = inputs.cavity_state(N, Ra, seed)
    state = dict(st, prev=None, steps=0)
    cav = H.Cavity(p)
    for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA),
                        ("p", H.HOSC_P)):
        cav.set(which, st[name])
    if history:
        old = inputs.perturbed(st, seed + 1000)
        lev = O.level_coefficients(dict(old, prev=None), op)
        prev = dict(L=lev["L"], u=old["u"], v=old["v"], w=old["w"], Eu=lev["Eu"], Ev=lev["Ev"],
                    Ew=lev["Ew"])
        state["prev"] = prev
        for key, which in (("L", H.HOSC_PREV_L), ("u", H.HOSC_PREV_U), ("v", H.HOSC_PREV_V),
                           ("w", H.HOSC_PREV_W), ("Eu", H.HOSC_PREV_EU), ("Ev", H.HOSC_PREV_EV),
                           ("Ew", H.HOSC_PREV_EW)):
            cav.set(which, prev[key])
    return p, op, state, cav


# (N, Ra, n, history, Ly, Lz): the cube, and boxes 1 x Ly x Lz with three different spacings
CASES = [(7, 1e3, 1.0, True, 1.0, 1.0), (13, 1e4, 0.75, True, 1.0, 1.0),
         (13, 5e3, 1.25, False, 1.0, 1.0), (22, 1e4, 0.8, True, 1.0, 1.0),
         (22, 2e3, 1.0, False, 1.0, 1.0), (13, 1e4, 0.75, True, 0.7, 1.4),
         (22, 5e3, 1.25, False, 1.6, 0.55)]


@pytest.mark.parametrize("N,Ra,n,history,Ly,Lz", CASES)
def test_stage_parity(N, Ra, n, history, Ly, Lz):
    p, op, state, cav = _setup(N, Ra, n, seed=N * 7 + int(n * 100), history=history, dt=0.004,
                               Ly=Ly, Lz=Lz)
    g = O.Grid.of(op)
    ii = g.int_idx
    with cav:
        # S1
        cav.run_stage(H.HOSC_STAGE_VISCOSITY)
        eta_o, _, gr = O.viscosity(state["u"], state["v"], state["w"], op)
        assert _rel(cav.get(H.HOSC_ETA), eta_o) < 1e-13
        assert _rel(cav.get(H.HOSC_LCOEF), 1.0 / (op.Pr * eta_o)) < 1e-13
        # S2
        cav.run_stage(H.HOSC_STAGE_SOURCES)
        Eu, Ev, Ew = O.momentum_sources(state["u"], state["v"], state["w"], state["th"],
                                        state["p"], eta_o, gr, op)
        for which, ref in ((H.HOSC_EU, Eu), (H.HOSC_EV, Ev), (H.HOSC_EW, Ew)):
            assert _rel(cav.get(which), ref) < 1e-12
        # S3
        cav.run_stage(H.HOSC_STAGE_RHS)
        lev = O.level_coefficients(state, op)
        coefs = O._system_coefficients(g, op, lev, state["prev"])
        rhs_o = {}
        for name, which in (("u", H.HOSC_RHS_U), ("v", H.HOSC_RHS_V), ("w", H.HOSC_RHS_W),
                            ("th", H.HOSC_RHS_THETA)):
            c = coefs[name]
            R = c["R"]
            Bx = O.apply_B(g, c, state[name].ravel())
            ref = (op.dt * (R - Bx))[ii]
            got = cav.get(which).ravel()[ii]
            scale = op.dt * max(np.max(np.abs(R[ii])), np.max(np.abs(Bx[ii])))
            assert np.max(np.abs(got - ref)) / scale < 1e-11, name
            rhs_o[name] = got
        # S4: the seven level-(n+1) weights of both operators, node by node
        A_m = O.assemble_A(g, op.dt, coefs["u"], op.a_limit, op.a_boost)
        A_e = O.assemble_A(g, op.dt, coefs["th"], op.a_limit, op.a_boost)
        offs = (0, 1, -1, N, -N, N * N, -N * N)
        for base, A in ((H.HOSC_A_MOM, A_m), (H.HOSC_A_ENE, A_e)):
            ref = np.stack([np.asarray(A[ii, ii + o]).ravel() for o in offs])
            got = np.stack([cav.get(base + q).ravel()[ii] for q in range(7)])
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), base
        # S5: GPU increment vs direct solve of the oracle operator; oracle A x_gpu = rhs_gpu
        info = cav.run_stage(H.HOSC_STAGE_SOLVE)
        assert info["status"] == 0
        import scipy.sparse.linalg as spla
        for name, which in (("u", H.HOSC_DX_U), ("v", H.HOSC_DX_V), ("w", H.HOSC_DX_W),
                            ("th", H.HOSC_DX_THETA)):
            A = (A_e if name == "th" else A_m)[ii][:, ii].tocsc()
            x_gpu = cav.get(which).ravel()[ii]
            b = rhs_o[name]
            assert np.linalg.norm(A @ x_gpu - b) <= 1e-11 * max(np.linalg.norm(b), 1e-300)
            x_ref = spla.spsolve(A, b)
            assert _rel(x_gpu, x_ref) < 1e-9, name
        # S6-S8: the full step against the oracle's step
        cav.run_stage(H.HOSC_STAGE_UPDATE)
        new, oinfo = O.step(state, op, g)
        for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                            ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
            assert _rel(cav.get(which), new[name]) < 1e-10, name
        div_o = O.divergence(new["u"], new["v"], new["w"], g.h, g.k, g.l)
        assert _rel(cav.get(H.HOSC_DIV).ravel()[ii], div_o.ravel()[ii]) < 1e-9


@pytest.mark.parametrize("N,n,hist,Ly,Lz", [(21, 1.0, 1, 1.0, 1.0), (21, 0.75, 1, 1.0, 1.0),
                                             (16, 1.25, 1, 1.0, 1.0), (17, 0.75, 0, 1.0, 1.0),
                                             (17, 0.75, 1, 0.8, 1.3)])
def test_trajectory_from_rest(N, n, hist, Ly, Lz):
    """Several steps from the initial state (fluid at rest), the configuration marched to
    steady state: fields, step change and divergence agree after every step (the cube and a
    box)."""
    p = _params(N, 1e3, n, dt=0.005, use_history=hist, Ly=Ly, Lz=Lz)
    op = _oracle_params(p)
    g = O.Grid.of(op)
    st = O.initial_state(op)
    with H.Cavity(p) as cav:
        assert _rel(cav.get(H.HOSC_THETA), st["th"]) == 0.0
        for _ in range(6):
            info = cav.step(1)
            st, oinfo = O.step(st, op, g)
            assert info["call_status"] == 0
            for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                                ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
                assert _rel(cav.get(which), st[name]) < 1e-10, name
            assert abs(info["res"] - oinfo["res"]) <= 1e-9 * oinfo["res"]
            assert abs(info["div_max"] - oinfo["div_max"]) <= 1e-9 * oinfo["div_max"]
            # iteration counts are decided by rounding near the tolerance; they agree closely
            for s, name in enumerate(("u", "v", "w", "th")):
                assert abs(info["last_iters"][s] - oinfo["iters"][name]) <= 2 + oinfo["iters"][name] // 10


def test_diagnostics_parity():
    for N, n, Ly, Lz in ((13, 0.75, 1.0, 1.0), (14, 1.0, 1.0, 1.0), (21, 1.25, 1.0, 1.0),
                         (13, 0.75, 0.6, 1.5), (14, 1.0, 1.8, 0.7)):
        p = _params(N, 1e4, n, Ly=Ly, Lz=Lz)
        op = _oracle_params(p)
        st = inputs.cavity_state(N, 1e4, seed=N)
        with H.Cavity(p) as cav:
            for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                                ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
                cav.set(which, st[name])
            d = cav.diagnostics(with_fields=True)
        o = O.diagnostics(st, op)
        for k_gpu, k_ora in (("Nu_hot_max", "Nu_hot_max"), ("Nu_hot_mean", "Nu_hot_mean"),
                             ("Nu_cold_mean", "Nu_cold_mean"), ("E_total", "E_total"),
                             ("E_HT", "E_HT_total"), ("E_FF", "E_FF_total"), ("Be", "Be")):
            assert d[k_gpu] == pytest.approx(o[k_ora], rel=1e-12, abs=1e-14), k_gpu
        assert _rel(d["Nu_avg_z"], o["Nu_avg_z"]) < 1e-12
        for k in ("E_HT", "E_FF", "E_local"):
            assert _rel(d[k + "_field"], o[k]) < 1e-12


def test_conduction_fixed_point_and_zero_rhs():
    """Ra = 0 with theta = 1 - x: the momentum right-hand sides are zero (no BiCGSTAB iteration),
    the state is unchanged to rounding and Nu = E_total = Be = 1."""
    N = 11
    p = _params(N, 0.0, 0.75)
    x = np.linspace(0, 1, N)
    th = np.broadcast_to(1.0 - x, (N, N, N)).copy()
    with H.Cavity(p) as cav:
        cav.set(H.HOSC_THETA, th)
        info = cav.step(2)
        # the velocity right-hand sides are exactly zero; theta's only carry rounding of 1 - x
        assert info["call_status"] == 0 and info["last_iters"][:3] == [0, 0, 0]
        assert info["res"] < 1e-13 and info["div_max"] == 0.0
        assert np.max(np.abs(cav.get(H.HOSC_THETA) - th)) < 1e-13
        assert np.max(np.abs(cav.get(H.HOSC_V))) == 0.0
        d = cav.diagnostics()
        for k in ("Nu_hot_max", "Nu_hot_mean", "Nu_cold_mean", "E_total", "Be"):
            assert d[k] == pytest.approx(1.0, abs=1e-12), k


def test_torch_workspace_matches_library_allocation():
    torch = pytest.importorskip("torch")
    p = _params(13, 1e4, 0.75)
    st = inputs.cavity_state(13, 1e4, seed=5)
    outs = []
    for ws in (None, "torch"):
        with H.Cavity(p, workspace=ws) as cav:
            for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                                ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
                cav.set(which, st[name])
            cav.step(3)
            outs.append([cav.get(w) for w in (H.HOSC_U, H.HOSC_V, H.HOSC_THETA, H.HOSC_P)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert torch.cuda.is_available()


def test_errors_and_limits():
    p = _params(9, 1e3, 1.0)
    p.max_lin_iter = 1
    st = inputs.cavity_state(9, 1e3, seed=2)
    with H.Cavity(p) as cav:
        cav.set(H.HOSC_V, st["v"])
        info = cav.step(1)
        assert info["call_status"] == H.HOSC_ENOCONV
        assert max(info["last_iters"]) == 1
        # stages out of order
        st_, _ = H.hosc_run_stage(cav.h, H.HOSC_STAGE_RHS)
        assert st_ == H.HOSC_ESTATE
        # read-only field, bad selector
        assert H.hosc_set_field(cav.h, H.HOSC_ETA, np.zeros((9, 9, 9))) == H.HOSC_EINVAL
        assert H.hosc_get_field(cav.h, 99, np.zeros((9, 9, 9))) == H.HOSC_EINVAL
    # a NaN in the state is reported as divergence, not hidden
    p = _params(9, 1e3, 1.0)
    with H.Cavity(p) as cav:
        u = st["u"].copy()
        u[4, 4, 4] = np.nan
        cav.set(H.HOSC_U, u)
        info = cav.step(1)
        assert info["call_status"] == H.HOSC_EDIVERGED
    bad = _params(9, 1e3, 1.0)
    bad.dt = -1.0
    st_, h = H.hosc_create(bad)
    assert st_ == H.HOSC_EINVAL and not h.value
    for Ly, Lz in ((-1.0, 1.0), (1.0, 100.0), (0.01, 1.0), (float("nan"), 1.0)):
        st_, h = H.hosc_create(_params(9, 1e3, 1.0, Ly=Ly, Lz=Lz))
        assert st_ == H.HOSC_EINVAL and not h.value, (Ly, Lz)


def test_small_and_even_grids():
    """N = 5 (one interior plane of 3^3) and even N (trapezoid diagnostics) against the oracle."""
    for N in (5, 6, 8):
        p = _params(N, 1e3, 0.9, dt=0.002)
        op = _oracle_params(p)
        st = O.initial_state(op)
        g = O.Grid(N)
        with H.Cavity(p) as cav:
            for _ in range(3):
                cav.step(1)
                st, _ = O.step(st, op, g)
            for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("th", H.HOSC_THETA),
                                ("p", H.HOSC_P)):
                assert _rel(cav.get(which), st[name]) < 1e-10, (N, name)
            d = cav.diagnostics()
        o = O.diagnostics(st, op)
        assert d["Nu_hot_mean"] == pytest.approx(o["Nu_hot_mean"], rel=1e-12)
        assert d["Be"] == pytest.approx(o["Be"], rel=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_captured_steps_match_stage_by_stage(precision):
    """hosc_step enqueues captured steps (BiCGSTAB as a device-side loop, no host round trip);
    with per-launch timing on, the same steps run stage by stage from the host. Same kernels in
    the same order: the fields must agree bit for bit, and so must the step records."""
    N = 17
    st = inputs.cavity_state(N, 1e4, seed=9)
    outs = []
    for timed in (False, True):
        p = _params(N, 1e4, 0.8, dt=0.002, precision=precision, tol_lin=1e-10)
        with H.Cavity(p) as cav:
            for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                                ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
                cav.set(which, st[name])
            H.hosc_profile_enable(cav.h, 1 if timed else 0)
            info = cav.step(5)
            outs.append((info, [cav.get(w) for w in (H.HOSC_U, H.HOSC_V, H.HOSC_W, H.HOSC_THETA,
                                                      H.HOSC_P)]))
    (ia, fa), (ib, fb) = outs
    assert ia["steps"] == ib["steps"] == 5 and ia["lin_iters"] == ib["lin_iters"]
    assert ia["res"] == ib["res"] and ia["div_max"] == ib["div_max"]
    for a, b in zip(fa, fb):
        assert np.array_equal(a, b)


def test_captured_steady_stop_is_exact():
    """solve_steady with captured steps stops on the device at the first steady step: the same
    step count and fields as the stage-by-stage solve."""
    N = 11
    res = []
    for timed in (False, True):
        p = _params(N, 1e3, 1.0, dt=0.02, tol_lin=1e-10, tol_steady=1e-4, tol_div=1e-3,
                    lambda_=0.1)
        with H.Cavity(p) as cav:
            H.hosc_profile_enable(cav.h, 1 if timed else 0)
            info = cav.solve_steady(5000)
            res.append((info, cav.get(H.HOSC_V)))
    (ia, va), (ib, vb) = res
    assert ia["call_status"] == ib["call_status"] == 0
    assert ia["steps"] == ib["steps"] and np.array_equal(va, vb)


def test_isolated_kernel_timing_leaves_the_state():
    """hosc_time_kernel re-runs one kernel class on the last step's buffers: positive times and
    bytes for every class, unchanged fields, and a following step equal to one taken without the
    timing (the Krylov buffers are re-initialised by every step)."""
    N = 15
    outs = []
    for timed in (False, True):
        p = _params(N, 1e4, 0.75, dt=0.002, tol_lin=1e-10)
        with H.Cavity(p) as cav:
            st = inputs.cavity_state(N, 1e4, seed=77)
            for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                                ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
                cav.set(which, st[name])
            cav.step(1)
            before = cav.get(H.HOSC_U)
            if timed:
                for kid in range(H.HOSC_K_BICG_XR + 1):
                    rc, ms, b = H.hosc_time_kernel(cav.h, kid, 5)
                    assert rc == 0 and ms > 0 and b > 0, (kid, rc, ms, b)
                assert np.array_equal(cav.get(H.HOSC_U), before)
                assert H.hosc_time_kernel(cav.h, H.HOSC_K_UPDATE, 5)[0] == H.HOSC_EINVAL
                assert H.hosc_time_kernel(cav.h, 0, 0)[0] == H.HOSC_EINVAL
            cav.step(1)
            outs.append(cav.get(H.HOSC_U))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", [H.HOSC_FP64, H.HOSC_MIXED])
def test_jacobi_row_scaling_one_step(precision):
    """With Jacobi row scaling (not in the paper) a step still gives the oracle's step: to 1e-10
    in FP64 (both solved to 1e-13 relative residual), and the increment to FP32 accuracy (2e-5
    of its size) in mixed precision."""
    N, Ra, n = 15, 1e4, 0.75
    p = _params(N, Ra, n, dt=0.002, precond=1, precision=precision)
    if precision == H.HOSC_MIXED:
        p.lambda_ = min(p.lambda_, 0.1)
    op = _oracle_params(p)
    st = inputs.cavity_state(N, Ra, seed=315)
    new, _ = O.step(dict(st, prev=None, steps=0), op, O.Grid(N))
    with H.Cavity(p) as cav:
        for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                            ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
            cav.set(which, st[name])
        info = cav.step(1)
        assert info["call_status"] == 0
        for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                            ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
            got = cav.get(which)
            if precision == H.HOSC_FP64:
                assert _rel(got, new[name]) <= 1e-10, name
            else:
                inc = new[name] - st[name]
                scale = max(np.max(np.abs(inc)), 1e-12)
                assert np.max(np.abs((got - st[name]) - inc)) <= 2e-5 * scale + 1e-12, name


FIELDS5 = (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA),
           ("p", H.HOSC_P))


@pytest.mark.parametrize("N,Ra,n,Ly,Lz", [(15, 1e4, 0.75, 1.0, 1.0), (12, 3e3, 1.25, 1.0, 1.0),
                                           (13, 1e4, 0.75, 0.8, 1.3)])
def test_bicgstab2_one_step(N, Ra, n, Ly, Lz):
    """BiCGSTAB(2) (solver = 1): one step equals the oracle's BiCGSTAB(2) step to 1e-10 (both
    solved to 1e-13), the iteration counts (two per cycle) agree with the oracle's, and the
    increments solve the oracle's operator: A x_gpu = rhs to 1e-11 of |rhs|."""
    p = _params(N, Ra, n, dt=0.002, solver=1, Ly=Ly, Lz=Lz)
    op = _oracle_params(p)
    st = inputs.cavity_state(N, Ra, seed=400 + N)
    g = O.Grid.of(op)
    new, oinfo = O.step(dict(st, prev=None, steps=0), op, g)
    assert oinfo["status"] == 0
    with H.Cavity(p) as cav:
        for name, which in FIELDS5:
            cav.set(which, st[name])
        info = cav.step(1)
        assert info["call_status"] == 0
        for name, which in FIELDS5:
            assert _rel(cav.get(which), new[name]) <= 1e-10, name
        for s_, name in enumerate(("u", "v", "w", "th")):
            it = info["last_iters"][s_]
            assert it % 2 == 0 and abs(it - oinfo["iters"][name]) <= 2, (name, it, oinfo["iters"])


def test_bicgstab2_stage_solve_and_limits():
    """Stage by stage with BiCGSTAB(2): the increments of S5 match a direct solve of the oracle's
    operator to 1e-9; the solver needs the FP64 solve; isolated Krylov timing is not offered."""
    import scipy.sparse.linalg as spla
    N, Ra, n = 13, 1e4, 0.75
    p, op, state, cav = _setup(N, Ra, n, seed=77, history=False, dt=0.004, solver=1)
    g = O.Grid.of(op)
    ii = g.int_idx
    with cav:
        cav.run_stage(H.HOSC_STAGE_VISCOSITY)
        cav.run_stage(H.HOSC_STAGE_SOURCES)
        cav.run_stage(H.HOSC_STAGE_RHS)
        rhs = {name: cav.get(which).ravel()[ii] for name, which in
               (("u", H.HOSC_RHS_U), ("v", H.HOSC_RHS_V), ("w", H.HOSC_RHS_W),
                ("th", H.HOSC_RHS_THETA))}
        info = cav.run_stage(H.HOSC_STAGE_SOLVE)
        assert info["status"] == 0
        lev = O.level_coefficients(state, op)
        coefs = O._system_coefficients(g, op, lev, None)
        A_m = O.assemble_A(g, op.dt, coefs["u"], op.a_limit, op.a_boost)
        A_e = O.assemble_A(g, op.dt, coefs["th"], op.a_limit, op.a_boost)
        for name, which in (("u", H.HOSC_DX_U), ("v", H.HOSC_DX_V), ("w", H.HOSC_DX_W),
                            ("th", H.HOSC_DX_THETA)):
            A = (A_e if name == "th" else A_m)[ii][:, ii].tocsc()
            x_ref = spla.spsolve(A, rhs[name])
            assert _rel(cav.get(which).ravel()[ii], x_ref) < 1e-9, name
        assert H.hosc_time_kernel(cav.h, H.HOSC_K_BICG_PV, 2)[0] == H.HOSC_EINVAL
    st_, h = H.hosc_create(_params(9, 1e3, 1.0, solver=1, precision=H.HOSC_MIXED))
    assert st_ == H.HOSC_EINVAL and not h.value
    st_, h = H.hosc_create(_params(9, 1e3, 1.0, solver=2))
    assert st_ == H.HOSC_EINVAL and not h.value


def test_bicgstab2_trajectory_captured():
    """Captured steps (the device-side loop runs two BiCGSTAB(2) cycles per pass) from rest
    follow the oracle's BiCGSTAB(2) trajectory to 1e-10 over several steps."""
    N = 17
    p = _params(N, 1e3, 0.75, dt=0.005, solver=1)
    op = _oracle_params(p)
    g = O.Grid.of(op)
    st = O.initial_state(op)
    with H.Cavity(p) as cav:
        for _ in range(3):
            info = cav.step(2)
            assert info["call_status"] == 0
            for _ in range(2):
                st, oinfo = O.step(st, op, g)
            for name, which in FIELDS5:
                assert _rel(cav.get(which), st[name]) < 1e-10, name


def test_inner_pressure_passes_match_the_oracle():
    """Inner pressure passes (Sec. 2.2's "previous pressure iteration": E* again with the
    corrected pressure, u, v, w solved again, div V, correction) reproduce the oracle's step
    in FP64 to 1e-10, with the same number of passes; the mixed path runs the same passes and
    stays within 1e-4 of the FP64 step (relative to each field's change)."""
    N, Ra, n = 13, 1e4, 0.75
    st = inputs.cavity_state(N, Ra, seed=413)
    names = (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA),
             ("p", H.HOSC_P))
    out = {}
    for precision in (H.HOSC_FP64, H.HOSC_MIXED):
        p = _params(N, Ra, n, dt=0.002, inner_max=12, precision=precision)
        p.lambda_ = min(p.lambda_, 0.1)
        with H.Cavity(p) as cav:
            for name, which in names:
                cav.set(which, st[name])
            info = cav.step(1)
            assert info["call_status"] == 0
            out[precision] = (info, {name: cav.get(which) for name, which in names})
    op = _oracle_params(_params(N, Ra, n, dt=0.002, inner_max=12))
    op.lam = min(op.lam, 0.1)
    ref, rinfo = O.step(dict(st, prev=None, steps=0), op, O.Grid(N))
    info64, f64 = out[H.HOSC_FP64]
    assert info64["inner_passes"] == rinfo["inner"] > 0
    for name, _ in names:
        assert _rel(f64[name], ref[name]) <= 1e-10, name
    infomx, fmx = out[H.HOSC_MIXED]
    assert infomx["inner_passes"] == rinfo["inner"]
    for name, _ in names:
        scale = max(np.max(np.abs(f64[name] - st[name])), 1e-12)
        assert np.max(np.abs(fmx[name] - f64[name])) <= 1e-4 * scale, name
    with pytest.raises(H.HoscError):
        H.Cavity(_params(N, Ra, n, inner_max=-1))
