"""The native pool (batching and serving): members advance together and give the same result
alone, in a mix, in either launch mode, and as a plain single-cavity solve; admission follows the
device-memory budget."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2411_06563_gb300.hosc")
from paper_2411_06563_gb300 import serve as S  # noqa: E402

FIELDS = (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA), ("p", H.HOSC_P))

# (N, Ra, n): the cavity followed by the tests, then the others of the mix
TARGET = (15, 2e3, 0.9)
OTHERS = [(11, 5e2, 1.2), (21, 1e3, 1.0), (13, 3e3, 0.8), (17, 1e3, 1.1), (9, 1e2, 1.0)]


def _params(N, Ra, n, precision=H.HOSC_MIXED):
    """Loose steady tolerances and a fixed dt = 0.01 (inside the stability bound at these Ra)
    keep the solves to a few thousand steps; FP32 sweeps throughout (no phase switch, whose step
    depends on when the host reads the records)."""
    p = S.request_params(N, Ra, n, precision=precision, tol_steady=1e-2, tol_div=1e-3)
    p.dt = 0.01
    p.lambda_ = 0.1
    p.auto_defect = 0
    return p


def _solve(members, mode=H.HOSC_POOL_GRAPH, autotune=False, G=8, max_steps=4000):
    """Run members to completion in one pool; results of all members, in order."""
    budget = sum(H.hosc_workspace_bytes(_params(*m)) for m in members) + 1
    with S.Pool(budget, G, mode, autotune) as pool:
        slots = [pool.admit(_params(*m), max_steps) for m in members]
        assert None not in slots
        out = {}
        while len(out) < len(members):
            for slot in pool.run(50):
                out[slot] = pool.result(slot, FIELDS)
        stats = pool.stats()
    return [out[s] for s in slots], stats


def test_same_alone_and_in_the_mix():
    alone, _ = _solve([TARGET])
    mixed, stats = _solve([TARGET] + OTHERS)
    a, b = alone[0], mixed[0]
    assert a["status"] == b["status"] == 0
    assert a["info"]["steps"] == b["info"]["steps"]
    for name, _ in FIELDS:
        assert np.array_equal(a[name], b[name]), name
    assert a["diag"] == b["diag"]
    # the others reach steady state or their step limit; none fails
    assert all(r["status"] in (0, H.HOSC_ESTEPLIMIT) for r in mixed), [r["status"] for r in mixed]
    assert stats["captures"] >= 2   # captured again as members completed


def test_graph_and_stream_modes_agree():
    g, _ = _solve([TARGET] + OTHERS[:2], mode=H.HOSC_POOL_GRAPH)
    s, stats = _solve([TARGET] + OTHERS[:2], mode=H.HOSC_POOL_STREAMS)
    assert stats["captures"] == 0
    for a, b in zip(g, s):
        assert a["status"] == b["status"] and a["info"]["steps"] == b["info"]["steps"]
        for name, _ in FIELDS:
            assert np.array_equal(a[name], b[name]), name


def test_pool_member_equals_plain_solve():
    """A member stops at the same first steady step as hosc_solve_steady on its own context."""
    res, _ = _solve([TARGET], G=6)
    with H.Cavity(_params(*TARGET)) as cav:
        info = cav.solve_steady(4000)
        assert info["call_status"] == 0
        assert info["steps"] == res[0]["info"]["steps"]
        for name, which in FIELDS:
            assert np.array_equal(cav.get(which), res[0][name]), name


def test_autotuned_mix_within_tolerance():
    """With the launch shape tuned per grid size the dot products group differently; the steady
    fields stay within the mixed-precision target (1e-5 max-abs) of the untuned run."""
    a, _ = _solve([TARGET] + OTHERS[:3], autotune=False)
    b, stats = _solve([TARGET] + OTHERS[:3], autotune=True)
    assert stats["tuned_sizes"] >= 1
    assert a[0]["status"] == b[0]["status"] == 0
    for name, _ in FIELDS[:4]:
        assert np.max(np.abs(a[0][name] - b[0][name])) <= 1e-5, name


def test_admission_by_budget():
    p = _params(13, 1e3, 1.0)
    need = H.hosc_workspace_bytes(p)
    with S.Pool(2 * need + 10, 4, H.HOSC_POOL_GRAPH, False) as pool:
        s0 = pool.admit(p, 10)
        s1 = pool.admit(p, 10)
        assert s0 is not None and s1 is not None and s0 != s1
        assert pool.admit(p, 10) is None          # no room now
        with pytest.raises(H.HoscError):
            pool.admit(_params(41, 1e3, 1.0), 10)  # never fits
        st = pool.stats()
        assert st["active"] == 2 and st["bytes_used"] <= st["budget"]
        done = pool.run(3)                         # 4 steps per round: 12 >= 10 steps
        assert sorted(done) == sorted([s0, s1])
        for s in done:
            r = pool.result(s)
            assert r["status"] == H.HOSC_ESTEPLIMIT and r["info"]["steps"] == 12
        pool.retire(s0)
        assert pool.admit(p, 10) is not None       # room again
    assert H.hosc_pool_create(0, 4, 0, 0)[0] == H.HOSC_EINVAL
    assert H.hosc_pool_create(1 << 20, 3, H.HOSC_POOL_GRAPH, 0)[0] == H.HOSC_EINVAL


# ------------------------------------------------------------- the persistent round kernel

def _round_tiles(N):
    """The Krylov launch shape of the persistent round kernel: 256-thread blocks, segments of
    eight planes (fewer on grids with fewer interior planes)."""
    return 256, min(N - 2, 8), 0


def test_persistent_round_matches_plain_solve():
    """A pool in persistent mode (one launch of the round kernel per round, all members' phases
    on one cooperative grid) runs the per-kernel path's device bodies tile for tile, so each
    member of a mix of sizes follows its plain single-cavity solve with the same launch shape:
    after 40 steps the fields agree within the FP32 rounding of the sweeps (1e-6 of each field's
    size: the two builds may contract a product and a sum into one fused multiply-add in
    different places), and the solves to the (loose) steady stop end with the same status within
    1 % of the steps."""
    members = [TARGET] + OTHERS[:4]
    fixed, _ = _solve(members, mode=H.HOSC_POOL_PERSISTENT, G=8, max_steps=40)
    res, stats = _solve(members, mode=H.HOSC_POOL_PERSISTENT, G=8)
    assert stats["captures"] == 0 and stats["rounds"] >= 1
    for m, f, r in zip(members, fixed, res):
        with H.Cavity(_params(*m)) as cav:
            assert H.hosc_set_tiles(cav.h, *_round_tiles(m[0])) == 0
            info = cav.step(40)
            assert f["status"] == H.HOSC_ESTEPLIMIT and f["info"]["steps"] == 40
            for name, which in FIELDS:
                a = cav.get(which)
                assert np.max(np.abs(a - f[name])) <= 1e-6 * max(1.0, np.max(np.abs(a))), (m, name)
        with H.Cavity(_params(*m)) as cav:
            assert H.hosc_set_tiles(cav.h, *_round_tiles(m[0])) == 0
            info = cav.solve_steady(4000, allow=(H.HOSC_ESTEPLIMIT, H.HOSC_ENOCONV))
            assert info["call_status"] == r["status"], (m, info, r["status"])
            assert abs(info["steps"] - r["info"]["steps"]) <= 0.01 * info["steps"] + 2, m


def test_persistent_round_admission():
    """The round kernel runs mixed-precision BiCGSTAB members without history terms: anything
    else is refused at admission."""
    with S.Pool(1 << 30, 8, H.HOSC_POOL_PERSISTENT, False) as pool:
        with pytest.raises(H.HoscError):
            pool.admit(_params(13, 1e3, 1.0, precision=H.HOSC_FP64), 10)
        p = _params(13, 1e3, 1.0)
        p.use_history = 1
        with pytest.raises(H.HoscError):
            pool.admit(p, 10)
        s = pool.admit(_params(13, 1e3, 1.0), 10)
        assert s is not None
        done = pool.run(2)
        assert done == [s]
        assert pool.result(s)["status"] == H.HOSC_ESTEPLIMIT
    assert H.hosc_pool_create(1 << 20, 8, 3, 0)[0] == H.HOSC_EINVAL
