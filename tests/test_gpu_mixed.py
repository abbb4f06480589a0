"""Mixed precision (FP32 sweeps and Krylov vectors; FP64 state, reductions, pressure update and
diagnostics) against the FP64 oracle and the FP64 GPU path.

Targets: fields within 1e-5 max-abs and Nu_avg within 1e-4 relative of FP64 at steady state; one
step from a seeded state within FP32 rounding of the increment.
"""

import numpy as np
import pytest

from oracle import hosc_oracle as O

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2411_06563_gb300.hosc")
from paper_2411_06563_gb300 import inputs  # noqa: E402

FIELDS = (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA), ("p", H.HOSC_P))


def _params(N, Ra, n, dt, precision, **kw):
    p = H.hosc_default_params(N, Ra, 1.0, n)
    p.dt = dt
    p.lambda_ = min(0.25 / (N - 1) ** 2 / dt, 0.1)
    p.precision = precision
    p.max_lin_iter = 3000
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("N,Ra,n,Ly,Lz", [(13, 1e4, 0.75, 1.0, 1.0), (22, 2e3, 1.0, 1.0, 1.0),
                                           (17, 5e3, 1.25, 1.0, 1.0), (17, 5e3, 0.75, 0.7, 1.5)])
def test_one_step_from_seeded_state(N, Ra, n, Ly, Lz):
    """One mixed step against the oracle's FP64 step from a seeded (far from steady) state: the
    increment chi^{n+1} - chi^n agrees to FP32 accuracy, 2e-5 relative to its size in the cube.
    The FP32 solve stops at a relative residual of 3e-6, and the error of the increment is that
    residual times the operator's conditioning, which the unequal spacings of a box raise (here
    k : l = 1 : 2.1): 5e-5 there (2.5e-5 measured)."""
    tol = 2e-5 if (Ly, Lz) == (1.0, 1.0) else 5e-5
    dt = 0.002
    p = _params(N, Ra, n, dt, H.HOSC_MIXED, tol_lin=1e-12, Ly=Ly, Lz=Lz)
    op = O.Params(N=N, Ra=Ra, n=n, dt=dt, lam=p.lambda_, tol_lin=1e-12, a_limit=p.a_limit,
                  a_boost=p.a_boost, Ly=Ly, Lz=Lz)
    st = inputs.cavity_state(N, Ra, seed=100 + N)
    g = O.Grid.of(op)
    new, _ = O.step(dict(st, prev=None, steps=0), op, g)
    with H.Cavity(p) as cav:
        for name, which in FIELDS:
            cav.set(which, st[name])
        info = cav.step(1)
        assert info["call_status"] == 0
        for name, which in FIELDS:
            got = cav.get(which)
            inc_ref = new[name] - st[name]
            scale = max(np.max(np.abs(inc_ref)), 1e-12)
            assert np.max(np.abs((got - st[name]) - inc_ref)) <= tol * scale + 1e-12, name


def _steady(p, max_steps):
    with H.Cavity(p) as cav:
        info = cav.solve_steady(max_steps)
        phase = H.hosc_get_phase(cav.h)
        fields = {name: cav.get(which) for name, which in FIELDS}
        d = cav.diagnostics()
    return info, phase, fields, d


def test_steady_state_matches_fp64():
    """Newtonian 21^3, Ra = 1e3 (the first configuration): the mixed solve (FP32 sweeps until the
    step change stalls, then FP64 defect sweeps) reaches the FP64 steady state: fields within
    1e-5 max-abs, Nu within 1e-4 relative, and the oracle's dt-free steady residual B chi - R of
    the mixed fields is as small as that of the FP64 fields."""
    N, dt = 21, 0.02
    kw = dict(tol_steady=1e-7, tol_div=1e-6, lambda_=0.1)
    i64, _, f64, d64 = _steady(_params(N, 1e3, 1.0, dt, H.HOSC_FP64, **kw), 20000)
    imx, phase, fmx, dmx = _steady(_params(N, 1e3, 1.0, dt, H.HOSC_MIXED, **kw), 20000)
    assert i64["call_status"] == 0 and imx["call_status"] == 0, (i64, imx)
    assert phase == 1   # the switch to FP64 defect sweeps happened
    for name, _ in FIELDS[:4]:
        assert np.max(np.abs(fmx[name] - f64[name])) <= 1e-5, name
    for k in ("Nu_hot_max", "Nu_hot_mean", "Nu_cold_mean"):
        assert abs(dmx[k] - d64[k]) <= 1e-4 * abs(d64[k]), k
    prm = O.Params(N=N, Ra=1e3, n=1.0, dt=dt)
    cert_mx, div_mx = O.steady_certificate(dict(fmx, prev=None), prm)
    cert_64, div_64 = O.steady_certificate(dict(f64, prev=None), prm)
    assert cert_mx <= max(10 * cert_64, 1e-5) and div_mx < 1e-6


def test_phase_api():
    p = _params(9, 1e3, 1.0, 0.01, H.HOSC_MIXED)
    with H.Cavity(p) as cav:
        assert H.hosc_get_phase(cav.h) == 0
        cav.step(2)
        assert H.hosc_set_phase(cav.h, 1) == 0 and H.hosc_get_phase(cav.h) == 1
        info = cav.step(2)
        assert info["call_status"] == 0
        assert H.hosc_set_phase(cav.h, 2) == H.HOSC_EINVAL
    p = _params(9, 1e3, 1.0, 0.01, H.HOSC_FP64)
    with H.Cavity(p) as cav:
        assert H.hosc_set_phase(cav.h, 1) == H.HOSC_EINVAL
        assert H.hosc_set_phase(cav.h, 0) == 0


def _one_mixed_step(N, Ra, n, dt, seed, tiles=None, stencil=None, merged=None, tma=None,
                    xr=None):
    p = _params(N, Ra, n, dt, H.HOSC_MIXED, tol_lin=1e-12)
    st = inputs.cavity_state(N, Ra, seed=seed)
    with H.Cavity(p) as cav:
        if merged is not None:
            assert H.hosc_set_krylov_merged(cav.h, merged) == 0
            assert H.hosc_get_krylov_merged(cav.h) == merged
        if tiles is not None:
            assert H.hosc_set_tiles(cav.h, *tiles) == 0
            assert H.hosc_get_tiles(cav.h)[:3] == (0,) + tuple(tiles[:2])
        if stencil is not None:
            assert H.hosc_set_stencil_tiles(cav.h, *stencil) == 0
            assert H.hosc_get_stencil_tiles(cav.h) == (0,) + tuple(stencil)
        if tma is not None:
            full = tuple(tma) + (3,) * (4 - len(tma))   # rows, planes, stages, kernels
            assert H.hosc_set_tma_tiles(cav.h, *full) == 0
            assert H.hosc_get_tma_tiles(cav.h) == (0,) + full
            assert H.hosc_get_stencil_tiles(cav.h) == (0, 0, 0, 0)
        if xr is not None:
            assert H.hosc_set_xr_form(cav.h, xr) == 0 and H.hosc_get_xr_form(cav.h) == xr
        for name, which in FIELDS:
            cav.set(which, st[name])
        info = cav.step(1)
        assert info["call_status"] == 0
        return p, st, {name: cav.get(which) - st[name] for name, which in FIELDS}


@pytest.mark.parametrize("tiles,merged", [((64, 1), 1), ((128, 3), 1), ((256, 17), 1),
                                          ((96, 7, 1), 1), ((256, 16, 1), 1), ((384, 17), 0),
                                          ((128, 5, 1), 0), ((160, 9), 0)])
def test_one_step_any_launch_shape(tiles, merged):
    """The launch shape of the interleaved FP32 solve (threads per block, planes per thread,
    register budget) and its form (two merged kernels per BiCGSTAB iteration, or three) change
    only the grouping of the float-float dot-product sums and the rounding of the recurrences:
    the increment equals the default's within the FP32 solve tolerance (relative residual
    3e-6), for segments that do not divide the interior, blocks that overhang the plane and a
    single segment. A missed or doubled plane or column would differ at O(1)."""
    N, Ra, n, dt = 19, 1e4, 0.75, 0.002
    _, _, ref = _one_mixed_step(N, Ra, n, dt, 219)
    _, _, got = _one_mixed_step(N, Ra, n, dt, 219, tiles, merged=merged)
    for name in ref:
        scale = max(np.max(np.abs(ref[name])), 1e-12)
        assert np.max(np.abs(got[name] - ref[name])) <= 1e-5 * scale, (name, tiles)


@pytest.mark.parametrize("stencil", [(32, 4, 9), (16, 2, 1), (8, 8, 17), (64, 4, 5), (24, 4, 3)])
def test_staged_stencil_kernels(stencil):
    """The staged (cp.async) p/v and s/t kernels compute what the register kernels compute: the
    increment equals the default's within the FP32 solve tolerance, for tiles that overhang the
    interior in x and y, single-plane and whole-column segments."""
    N, Ra, n, dt = 19, 1e4, 0.75, 0.002
    _, _, ref = _one_mixed_step(N, Ra, n, dt, 219)
    _, _, got = _one_mixed_step(N, Ra, n, dt, 219, stencil=stencil, merged=0)
    for name in ref:
        scale = max(np.max(np.abs(ref[name])), 1e-12)
        assert np.max(np.abs(got[name] - ref[name])) <= 1e-5 * scale, (name, stencil)


@pytest.mark.parametrize("tma", [(1, 1, 3), (2, 5, 4), (3, 17, 3), (4, 9, 6), (8, 3, 8),
                                 (17, 2, 3), (1, 17, 8), (2, 7, 6), (2, 9, 6, 1), (3, 5, 4, 2)])
def test_tma_stencil_kernels(tma):
    """The bulk-copy (TMA) p/v and s/t kernels compute what the register kernels compute: the
    increment equals the default's within the FP32 solve tolerance, for row tiles that overhang
    the interior in y (17 = 2 x 8 + 1, 3 x 5 + 2, ...), segments that do not divide the interior,
    single-plane and whole-column segments, a single tile per plane, rings of 3, 4, 6 and 8
    stages (segments shorter and longer than the ring), and either kernel alone beside the
    register form of the other."""
    N, Ra, n, dt = 19, 1e4, 0.75, 0.002
    _, _, ref = _one_mixed_step(N, Ra, n, dt, 219)
    _, _, got = _one_mixed_step(N, Ra, n, dt, 219, tma=tma, merged=0)
    for name in ref:
        scale = max(np.max(np.abs(ref[name])), 1e-12)
        assert np.max(np.abs(got[name] - ref[name])) <= 1e-5 * scale, (name, tma)


@pytest.mark.parametrize("N,tma", [(19, None), (19, (2, 5, 4)), (12, None), (31, (3, 7, 6, 1))])
def test_flat_xr_kernel(N, tma):
    """The flat x/r stream (every node of the interior planes, walls included) computes what the
    column march computes, alone and with the bulk-copy stencil kernels: the increment equals the
    default's within the FP32 solve tolerance."""
    Ra, n, dt = 1e4, 0.75, 0.002
    _, _, ref = _one_mixed_step(N, Ra, n, dt, 219)
    _, _, got = _one_mixed_step(N, Ra, n, dt, 219, tma=tma, merged=0, xr=1)
    for name in ref:
        scale = max(np.max(np.abs(ref[name])), 1e-12)
        assert np.max(np.abs(got[name] - ref[name])) <= 1e-5 * scale, (name, N, tma)


def test_tma_steps_and_shape_switches():
    """Captured steps with the bulk-copy kernels, then a switch to the staged kernels (which
    clears the bulk-copy shape) and back: every state equals the register kernels' run within the
    FP32 solve tolerance after each leg."""
    N, Ra, n, dt = 21, 1e4, 0.75, 0.002
    p = _params(N, Ra, n, dt, H.HOSC_MIXED, tol_lin=1e-10)
    st = inputs.cavity_state(N, Ra, seed=5)
    runs = []
    for plan in ("register", "switch"):
        with H.Cavity(p) as cav:
            for name, which in FIELDS:
                cav.set(which, st[name])
            out = []
            for leg in range(3):
                if plan == "switch":
                    if leg == 1:
                        assert H.hosc_set_stencil_tiles(cav.h, 16, 2, 5) == 0
                        assert H.hosc_get_tma_tiles(cav.h) == (0, 0, 0, 3, 3)
                    else:
                        assert H.hosc_set_tma_tiles(cav.h, 2, 6, 4, 3) == 0
                        assert H.hosc_get_stencil_tiles(cav.h) == (0, 0, 0, 0)
                info = cav.step(4)
                assert info["call_status"] == 0, info
                out.append(cav.get(H.HOSC_U))
            runs.append(out)
    for a, b in zip(*runs):
        assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(a)), "state after a leg"


def test_tiles_limits_and_autotune():
    N = 21
    p = _params(N, 1e4, 0.75, 0.002, H.HOSC_MIXED)
    with H.Cavity(p) as cav:
        for bad in ((32, 1), (100, 1), (512, 1), (128, 0), (128, N - 1), (384, 1, 1),
                    (128, 1, 2)):
            assert H.hosc_set_tiles(cav.h, *bad) == H.HOSC_EINVAL, bad
        for bad in ((4, 4, 1), (32, 16, 1), (32, 4, 0), (32, 4, N - 1), (64, 8, 1), (17, 2, 1)):
            assert H.hosc_set_stencil_tiles(cav.h, *bad) == H.HOSC_EINVAL, bad
        assert H.hosc_set_stencil_tiles(cav.h, 0, 0, 0) == 0
        for bad in ((1, 0, 3, 3), (1, N - 1, 3, 3), (N - 1, 1, 3, 3), (-1, 3, 3, 3),
                    (2, -4, 3, 3), (2, 4, 5, 3), (2, 4, 2, 3), (2, 4, 16, 3), (2, 4, 3, 0),
                    (2, 4, 3, 4)):
            assert H.hosc_set_tma_tiles(cav.h, *bad) == H.HOSC_EINVAL, bad
        assert H.hosc_set_tma_tiles(cav.h, 0, 5, 7, 1) == 0
        assert H.hosc_get_tma_tiles(cav.h) == (0, 0, 0, 3, 3)
        assert H.hosc_set_xr_form(cav.h, 2) == H.HOSC_EINVAL and H.hosc_get_xr_form(cav.h) == 0
        assert H.hosc_get_krylov_merged(cav.h) == 0   # the default form: three kernels
        assert H.hosc_set_krylov_merged(cav.h, 2) == H.HOSC_EINVAL
        assert H.hosc_set_tiles(cav.h, 384, 1) == 0
        assert H.hosc_set_krylov_merged(cav.h, 1) == H.HOSC_EINVAL   # 384 threads
        assert H.hosc_set_tiles(cav.h, 128, 1) == 0 and H.hosc_set_krylov_merged(cav.h, 1) == 0
        assert H.hosc_set_tiles(cav.h, 320, 1) == H.HOSC_EINVAL      # merged: at most 256
        assert H.hosc_set_krylov_merged(cav.h, 0) == 0
        cav.step(2)
        u0 = cav.get(H.HOSC_U)
        rc, b, z, ms = H.hosc_autotune(cav.h, 2)
        assert rc == 0 and b in (64, 96, 128, 160, 192, 256, 320, 384) and 1 <= z <= N - 2 and ms > 0
        assert H.hosc_get_tiles(cav.h)[:3] == (0, b, z)
        assert np.array_equal(cav.get(H.HOSC_U), u0)   # tuning leaves the state alone
        info = cav.step(3)
        assert info["call_status"] == 0
    p64 = _params(N, 1e4, 0.75, 0.002, H.HOSC_FP64)
    with H.Cavity(p64) as cav:
        cav.step(1)
        assert H.hosc_autotune(cav.h, 1)[0] == H.HOSC_EINVAL


def test_interleaved_fields_read_back():
    """In mixed precision the right-hand sides live in an interleaved float array and the two
    level-(n+1) operators in compact float form (per node the diagonal, the antisymmetric halves
    B_d of each direction, and L, from which the symmetric halves follow); hosc_get_field
    returns each right-hand side and each of the 14 weights as its own N^3 array. With FP64
    sweeps (phase 1) the right-hand sides are the FP64 path's values rounded once to float
    (within 2^-24 of each value) and every weight is the FP64 weight within a few float roundings
    of its row's largest weight (2^-21)."""
    N = 13
    st = inputs.cavity_state(N, 1e4, seed=31)
    got = {}
    for prec in (H.HOSC_FP64, H.HOSC_MIXED):
        p = _params(N, 1e4, 0.75, 0.002, prec)
        with H.Cavity(p) as cav:
            if prec == H.HOSC_MIXED:
                assert H.hosc_set_phase(cav.h, 1) == 0
            for name, which in FIELDS:
                cav.set(which, st[name])
            for stage in range(3):
                cav.run_stage(stage)
            got[prec] = {w: cav.get(w) for w in
                         [H.HOSC_RHS_U + s for s in range(4)] +
                         [H.HOSC_A_MOM + q for q in range(7)] +
                         [H.HOSC_A_ENE + q for q in range(7)]}
    rows = {}
    for base in (H.HOSC_A_MOM, H.HOSC_A_ENE):
        rows[base] = np.max(np.abs(np.stack([got[H.HOSC_FP64][base + q] for q in range(7)])), axis=0)
    for w, ref in got[H.HOSC_FP64].items():
        if w < H.HOSC_A_MOM:
            tol = 2.0 ** -24 * np.abs(ref) + 1e-37
        else:
            tol = 2.0 ** -21 * rows[H.HOSC_A_ENE if w >= H.HOSC_A_ENE else H.HOSC_A_MOM]
        assert np.all(np.abs(got[H.HOSC_MIXED][w] - ref) <= tol), w
