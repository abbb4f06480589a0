"""Batching and serving on top of the pool of libhosc.so (hosc_pool_* in include/hosc.h).

The pool (native) advances many cavity solves together, one round of captured steps per member
at a time, and completes each member when it is steady, failed or out of steps. This module
sets each request's parameters, drives the pool for a fixed batch, and runs the serving
loop: requests arrive on a (simulated) clock, wait in FIFO order until the device-memory budget
admits them, advance with everything else on the GPU, and leave when they complete; the loop
reports solves/s and percentiles of arrival-to-completion time.

The loop only talks to a pool object (``admit`` / ``run`` / ``result`` / ``retire``) and a clock,
so its bookkeeping is tested on the CPU with a stand-in pool.
"""

import math
import time

import numpy as np

from . import hosc as H


def request_params(N, Ra, n, Pr=1.0, precision=None, tol_steady=1e-6, tol_div=None):
    """hosc_params for one cavity solve of a batch or a request stream: the library's steady-solve
    rule (hosc_steady_params: pseudo-time step from the stability estimate of the scheme and the
    pressure relaxation, lambda = 2 Pr min(1, 2 eta_bl), no delta_t^- history), linear tolerance
    1e-10, mixed precision by default (FP32 sweeps, FP64 defect sweeps once the step change
    stalls)."""
    p = H.hosc_steady_params(N, Ra, Pr, n)
    p.tol_lin = 1e-10
    # the steady rule ties the correction threshold tol_div to tol_steady (h / (2 lambda)) and
    # stops at max|div V| < tol_steady; an explicit tol_div is both (the paper's one threshold)
    if tol_div is None:
        p.tol_div = p.tol_div * tol_steady / p.tol_steady
        p.div_steady = tol_steady
    else:
        p.tol_div = tol_div
        p.div_steady = 0.0
    p.tol_steady = tol_steady
    p.precision = H.HOSC_MIXED if precision is None else precision
    return p


class Pool:
    """The native pool as a Python object (see hosc_pool_* in include/hosc.h)."""

    def __init__(self, budget_bytes, steps_per_round=8, mode=H.HOSC_POOL_GRAPH, autotune=True):
        st, self.h = H.hosc_pool_create(budget_bytes, steps_per_round, mode, 1 if autotune else 0)
        if st:
            raise H.HoscError(st, "hosc_pool_create")
        self.budget = budget_bytes

    def admit(self, params, max_steps):
        """Slot index, or None when the budget has no room now. Raises for a request that can
        never fit or an error."""
        st, slot = H.hosc_pool_admit(self.h, params, max_steps)
        if st == H.HOSC_ENOMEM:
            return None
        if st:
            raise H.HoscError(st, "hosc_pool_admit")
        return slot

    def run(self, rounds=1):
        st, done = H.hosc_pool_run(self.h, rounds)
        if st:
            raise H.HoscError(st, "hosc_pool_run")
        return done

    def result(self, slot, fields=()):
        st, status, info, diag, ctx = H.hosc_pool_result(self.h, slot)
        if st:
            raise H.HoscError(st, "hosc_pool_result")
        out = dict(status=status, info=info.as_dict(), diag=diag.as_dict())
        if fields:
            _, p = H.hosc_get_params(ctx)
            N = p.N
            for name, which in fields:
                a = np.empty((N, N, N))
                rc = H.hosc_get_field(ctx, which, a)
                if rc:
                    raise H.HoscError(rc, "hosc_get_field")
                out[name] = a
        return out

    def retire(self, slot):
        st = H.hosc_pool_retire(self.h, slot)
        if st:
            raise H.HoscError(st, "hosc_pool_retire")

    def stats(self):
        _, s = H.hosc_pool_stats(self.h)
        return s.as_dict()

    def close(self):
        if self.h:
            H.hosc_pool_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def percentile(values, q):
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    if not values:
        return None
    return float(np.percentile(np.asarray(values, dtype=float), q))


def serve(requests, pool, make_params, max_steps, clock=time.perf_counter, sleep=time.sleep,
          rounds_per_poll=1, fields=()):
    """Serve a stream of requests (dicts with arrival time 't' in seconds from the start, and
    whatever make_params needs) on a pool.

    Continuous batching: at every poll the loop admits, in arrival order, every request that has
    arrived while the budget has room (a request that does not fit waits, and so does every later
    one: FIFO), runs the pool for rounds_per_poll rounds (returning early when a member
    completes), and retires completed members. Returns (results, summary): results[i] holds the
    request's admission and completion times, status, steps and diagnostics; the summary has
    solves/s (completed requests over the span from the first arrival to the last completion)
    and the p50 / p99 of arrival-to-completion time."""
    t0 = clock()
    pending = sorted(range(len(requests)), key=lambda i: requests[i]["t"])
    queue = []           # arrived, not admitted
    active = {}          # slot -> request index
    results = [None] * len(requests)
    nxt = 0
    while nxt < len(pending) or queue or active:
        now = clock() - t0
        while nxt < len(pending) and requests[pending[nxt]]["t"] <= now:
            queue.append(pending[nxt])
            nxt += 1
        while queue:
            i = queue[0]
            slot = pool.admit(make_params(requests[i]), max_steps)
            if slot is None:
                break
            queue.pop(0)
            active[slot] = i
            results[i] = dict(t_arrival=requests[i]["t"], t_admit=now)
        if not active:
            if nxt < len(pending):   # idle until the next arrival
                sleep(max(0.0, requests[pending[nxt]]["t"] - (clock() - t0)))
                continue
            if queue:
                raise RuntimeError("request %d can never be admitted" % queue[0])
            break
        done = pool.run(rounds_per_poll)
        t_done = clock() - t0
        for slot in done:
            i = active.pop(slot)
            r = pool.result(slot, fields)
            results[i].update(t_done=t_done, latency=t_done - results[i]["t_arrival"],
                              status=r["status"], steps=r["info"]["steps"],
                              lin_iters=r["info"]["lin_iters"], diag=r["diag"],
                              **{k: v for k, v in r.items() if k not in ("status", "info", "diag")})
            pool.retire(slot)
    lat = [r["latency"] for r in results if r is not None and "latency" in r]
    first = min(r["t"] for r in requests) if requests else 0.0
    last = max((r["t_done"] for r in results if r is not None and "t_done" in r), default=first)
    span = max(last - first, 1e-12)
    summary = dict(requests=len(requests), completed=len(lat),
                   steady=sum(1 for r in results if r and r.get("status") == H.HOSC_OK),
                   solves_per_s=len(lat) / span, span_s=span,
                   p50_s=percentile(lat, 50), p99_s=percentile(lat, 99),
                   mean_s=float(np.mean(lat)) if lat else None)
    return results, summary
