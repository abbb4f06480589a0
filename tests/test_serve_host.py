"""Host logic of the serving loop and the steady-solve parameter rule, on the CPU with a stand-in
pool and a simulated clock (the native pool itself is exercised by tests/test_gpu_pool.py)."""

import math

import numpy as np
import pytest

from paper_2411_06563_gb300 import inputs
from paper_2411_06563_gb300 import serve as S


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class FakePool:
    """Members need `work` rounds each; a round costs `round_s` seconds of the fake clock whatever
    the membership (a saturated device would not, but the bookkeeping is what is tested)."""

    def __init__(self, budget, clock, round_s=0.01):
        self.budget, self.clock, self.round_s = budget, clock, round_s
        self.used = 0
        self.members = {}
        self.next_slot = 0
        self.max_used = 0
        self.admitted = []

    def admit(self, params, max_steps):
        need = params["bytes"]
        if need > self.budget:
            raise RuntimeError("never fits")
        if self.used + need > self.budget:
            return None
        slot = self.next_slot
        self.next_slot += 1
        self.members[slot] = dict(left=params["work"], bytes=need, done=False, rounds=0,
                                  id=params["id"])
        self.used += need
        self.max_used = max(self.max_used, self.used)
        self.admitted.append(params["id"])
        return slot

    def run(self, rounds=1):
        done = []
        for _ in range(rounds):
            self.clock.t += self.round_s
            for slot, m in self.members.items():
                if not m["done"]:
                    m["left"] -= 1
                    m["rounds"] += 1
                    if m["left"] <= 0:
                        m["done"] = True
                        done.append(slot)
            if done:
                break
        return done

    def result(self, slot, fields=()):
        m = self.members[slot]
        return dict(status=0, info=dict(steps=8 * m["rounds"], lin_iters=0),
                    diag=dict(id=m["id"]))

    def retire(self, slot):
        self.used -= self.members.pop(slot)["bytes"]


def _requests(n, rate, seed=5):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return [dict(t=float(t[i]), id=i, bytes=int(rng.integers(1, 4)), work=int(rng.integers(1, 6)))
            for i in range(n)]


def test_every_request_completes_within_budget_fifo():
    clock = FakeClock()
    pool = FakePool(budget=6, clock=clock)
    reqs = _requests(60, rate=40.0)
    res, summ = S.serve(reqs, pool, lambda r: r, max_steps=100, clock=clock, sleep=clock.sleep)
    assert summ["completed"] == 60 and summ["steady"] == 60
    assert pool.max_used <= 6 and pool.used == 0 and not pool.members
    assert pool.admitted == sorted(pool.admitted)   # admission in arrival order
    for r, q in zip(res, reqs):
        assert r["diag"]["id"] == q["id"]
        assert r["t_arrival"] <= r["t_admit"] <= r["t_done"]
        assert r["latency"] == pytest.approx(r["t_done"] - q["t"])
        # a request needs at least its own rounds after admission
        assert r["t_done"] - r["t_admit"] >= q["work"] * 0.01 - 1e-9
    lat = sorted(r["latency"] for r in res)
    assert summ["p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert summ["p99_s"] == pytest.approx(np.percentile(lat, 99))
    span = max(r["t_done"] for r in res) - reqs[0]["t"]
    assert summ["solves_per_s"] == pytest.approx(60 / span)


def test_idle_loop_waits_for_arrivals():
    clock = FakeClock()
    pool = FakePool(budget=10, clock=clock)
    reqs = [dict(t=5.0, id=0, bytes=1, work=2), dict(t=9.0, id=1, bytes=1, work=1)]
    res, summ = S.serve(reqs, pool, lambda r: r, max_steps=10, clock=clock, sleep=clock.sleep)
    assert res[0]["t_admit"] == pytest.approx(5.0) and res[1]["t_admit"] == pytest.approx(9.0)
    assert res[0]["latency"] == pytest.approx(0.02) and res[1]["latency"] == pytest.approx(0.01)


def test_oversized_request_is_reported():
    clock = FakeClock()
    pool = FakePool(budget=2, clock=clock)
    with pytest.raises(RuntimeError):
        S.serve([dict(t=0.0, id=0, bytes=3, work=1)], pool, lambda r: r, max_steps=10,
                clock=clock, sleep=clock.sleep)


def test_percentile_definition():
    assert S.percentile([], 50) is None
    assert S.percentile([1.0, 2.0, 3.0, 4.0], 50) == pytest.approx(2.5)
    assert S.percentile([1.0] * 99 + [100.0], 99) == pytest.approx(1.99)


def test_steady_params_rule():
    """hosc_steady_params (host-only): dt keeps dt u^2 L <= 1 for the rule's velocity scale, is at
    most 0.02, and keeps lambda dt = 0.9 h^2 or below (the highest pressure mode); lambda is 2 Pr
    except in strongly shear-thinning flows; no delta_t^- history. The Newtonian 21^3 Ra = 1e3
    configuration gets lambda = 2 and dt = 0.45 h^2."""
    from paper_2411_06563_gb300 import hosc as H
    p = H.hosc_steady_params(21, 1e3, 1.0, 1.0)
    assert p.lambda_ == 2.0 and p.dt == pytest.approx(0.45 / 400.0, rel=1e-15)
    assert p.use_history == 0
    for N, Ra, n, Pr in [(41, 1e4, 0.75, 1.0), (101, 1e5, 0.75, 1.0), (61, 1e5, 1.25, 1.0),
                         (21, 1e2, 1.0, 1.0), (51, 1e4, 1.0, 0.71)]:
        p = H.hosc_steady_params(N, Ra, Pr, n)
        h = 1.0 / (N - 1)
        assert 0 < p.dt <= 0.02
        assert p.lambda_ * p.dt <= 0.9 * h * h * (1 + 1e-12)
        c = 0.12 * 2.0 ** (4 * (1 - n))
        u = max(1.0, 1.5 * c * math.sqrt(Ra))
        assert p.dt * u * u / Pr <= 1.0 + 1e-12   # L = 1/(Pr eta) >= 1/Pr only tightens it
        assert 0 < p.lambda_ <= 2.0 * Pr
        assert p.tol_div == pytest.approx(0.5 * p.tol_steady * h / p.lambda_, rel=1e-15)
        assert p.div_steady == p.tol_steady   # the stop tests the divergence at 1e-6
    # thinner fluids and faster flows need smaller steps
    dt = lambda N, Ra, n: H.hosc_steady_params(N, Ra, 1.0, n).dt
    assert dt(41, 1e5, 0.75) < dt(41, 1e5, 1.0)
    assert dt(21, 1e5, 1.0) < dt(21, 1e2, 1.0)
    assert H.hosc_steady_params(41, 1e4, 1.0, 0.75).lambda_ < 2.0
    with pytest.raises(H.HoscError):
        H.hosc_steady_params(21, -1.0, 1.0, 1.0)
    r = S.request_params(31, 1e3, 0.75)
    assert r.precision == H.HOSC_MIXED and r.tol_lin == 1e-10 and r.use_history == 0
    assert r.div_steady == r.tol_steady == 1e-6
    r = S.request_params(31, 1e3, 0.75, tol_steady=1e-4)
    q = H.hosc_steady_params(31, 1e3, 1.0, 0.75)
    assert r.div_steady == 1e-4 and r.tol_div == pytest.approx(100 * q.tol_div, rel=1e-15)
    r = S.request_params(31, 1e3, 0.75, tol_div=1e-3)
    assert r.tol_div == 1e-3 and r.div_steady == 0.0   # one threshold for both, as in Sec. 2.2
    assert H.hosc_default_params(21, 1e3, 1.0, 1.0).div_steady == 0.0


def test_batch_and_stream_recipes_are_seeded():
    a, b = inputs.batch_mix(), inputs.batch_mix()
    assert a == b and len(a) == 64
    assert {c["N"] for c in a} <= {21, 31, 41, 61}
    r = inputs.request_stream(50, rate=2.0)
    assert r == inputs.request_stream(50, rate=2.0)
    assert all(x["t"] <= y["t"] for x, y in zip(r, r[1:]))
