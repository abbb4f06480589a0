#!/usr/bin/env python
"""Benchmark of the HOSC pseudo-time step on GB300: grid-point updates per second (GPUPS).

One "step" is one pass of the whole hot path (viscosity, sources, compact right-hand sides,
BiCGSTAB on the four systems, walls, divergence and pressure correction, steady-state change)
over one cavity. GPUPS = (N - 2)^3 interior nodes x steps / second, summed over ranks.

Workload (default): the single large cavity of the headline configuration, 101^3 nodes,
n = 0.75, Ra = 1e5, Pr = 1, marched from rest (fluid at rest, theta = 1/2 inside) through a
spin-up before the timed steps. The working set (> 500 MB of device arrays) is larger than the
129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Pseudo-time step, relaxation and divergence tolerance of each workload: the library's
# steady-solve rule (hosc_steady_params; the timed steps are those of the steady solve). They are
# written out here so that the reference arm, which runs the oracle only, needs no part of the
# library; the GPU arm checks them against the library.
WORKLOADS = {
    "cavity101": dict(N=101, Ra=1e5, Pr=1.0, n=0.75, dt=1.1503218609060238e-05,
                      lam=0.5963268526936827, tol_div=8.384663506958269e-09, spinup=300,
                      history=0,
                      desc="single cavity 101^3, n=0.75, Ra=1e5, Pr=1 (power-law, shear-thinning), "
                           "mixed precision"),
    "cavity41": dict(N=41, Ra=1e4, Pr=1.0, n=0.75, dt=0.0001771411147115303,
                     lam=0.9182995386645731, tol_div=1.3612116170915195e-08, spinup=300,
                     history=0, desc="cavity 41^3, n=0.75, Ra=1e4, Pr=1, mixed precision"),
    # out-of-L2 probe: the Krylov working set (2 GB) is 15x the L2
    "cavity257": dict(N=257, Ra=1e5, Pr=1.0, n=0.75, dt=1.1503218609060238e-05,
                      lam=0.5963268526936827, tol_div=3.2752591824055733e-09, spinup=50,
                      history=0,
                      desc="single cavity 257^3, n=0.75, Ra=1e5, Pr=1, mixed precision "
                           "(out-of-L2 roofline probe)"),
}


# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum,
# mean of the captured launches) from ncu captures of the same kernel build, workload and launch
# shape, summarised under profiles/, over the launches of the uncaptured profiled steps (the
# in-step launches that `achieved` averages). Keyed by (workload, kernel class, launch shape as
# _kernel_shape gives it); any other configuration, or a kernel changed since its capture,
# reports null.
NCU_TRAFFIC = {
    # profiles/k4_pv_cavity101_mixed.md, "In-step DRAM traffic" (40 launches each)
    ("cavity101", "k_bicg_pv", ("register", 256, 9, 0)): 105.0e6,
    ("cavity101", "k_bicg_pv", ("register", 384, 9, 0)): 104.7e6,
    # profiles/k7_pv_bulk_copy_cavity101_mixed.md (50 in-step launches each)
    ("cavity101", "k_bicg_pv", ("bulk-copy", 2, 33, 6)): 96.2e6,
    ("cavity101", "k_bicg_st", ("register", 384, 9, 0)): 57.3e6,
    ("cavity101", "k_bicg_xr", ("flat",)): 98.7e6,
}


def _kernel_shape(kernel, shape):
    """The launch shape of a Krylov kernel class, as NCU_TRAFFIC keys it."""
    t, s, m = shape["tiles"], shape["stencil"], shape["tma"]
    reg = ("register", t["block"], t["kz"], t["narrow"])
    if kernel in ("k_bicg_pv", "k_bicg_st"):
        if m["rows"] and m["kernels"] & (1 if kernel == "k_bicg_pv" else 2):
            return ("bulk-copy", m["rows"], m["planes"], m["stages"])
        if s["sx"]:
            return ("staged", s["sx"], s["sy"], s["skz"])
        return reg
    if kernel == "k_bicg_xr":
        return ("flat",) if shape["xr"] == "flat stream" else reg
    return None


def _fp64_roofline(H, cav, N, steps=3):
    """The all-FP64 path's kernels against their two ceilings, over a few uncaptured steps: the
    BiCGSTAB kernels (p/v, s/t, x/r) as FP64 arithmetic, 32 fused multiply-adds per node, system
    and iteration (p/v: p update 2, operator 7, r_0 . v 1; s/t: s at the 7 stencil nodes 7,
    operator 7, two dot products 2; x/r: 4 updates, 2 dot products), against the FP64 FMA rate
    measured by hosc_fp64_peak, and as bytes against the measured copy bandwidth; the sweeps
    as bytes and time."""
    import torch
    names = ["k_viscosity", "k_sources", "k_rhs", "k_bicg_pv", "k_bicg_st", "k_bicg_xr", "update"]
    H.hosc_profile_enable(cav.h, 1)
    info = cav.step(steps)
    kern = {}
    for kid, name in enumerate(names):
        _, kms, kl, kb = H.hosc_profile_read(cav.h, kid)
        kern[name] = dict(ms=kms, launches=kl, bytes=kb)
    H.hosc_profile_enable(cav.h, 0)
    torch.cuda.synchronize()
    rc, tf = H.hosc_fp64_peak(20)
    peak, _ = _peaks()
    kry = sum(kern[k]["ms"] for k in ("k_bicg_pv", "k_bicg_st", "k_bicg_xr"))
    kry_b = sum(kern[k]["bytes"] for k in ("k_bicg_pv", "k_bicg_st", "k_bicg_xr"))
    flops = 64.0 * (N - 2) ** 3 * info["lin_iters"]
    out = {"steps": steps, "fp64_peak_tflops_measured": tf if rc == 0 else None,
           "krylov": {"ms_per_step": kry / steps,
                      "fp64_tflops": flops / (kry * 1e-3) / 1e12 if kry > 0 else None,
                      "GBps": kry_b / (kry * 1e-3) / 1e9 if kry > 0 else None},
           "kernels": {k: {"ms_per_step": v["ms"] / steps,
                           "GBps": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] else 0.0}
                       for k, v in kern.items()}}
    k = out["krylov"]
    k["fp64_frac"] = k["fp64_tflops"] / tf if (rc == 0 and tf > 0 and k["fp64_tflops"]) else None
    k["hbm_frac"] = k["GBps"] / peak if k["GBps"] else None
    return out


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for _, _, r in rows for q in range(4) if r[q].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def run_reference(args, wl):
    """The oracle (plain FP64 CPU implementation) timed on the host cores on the same workload:
    the same grid, physics, pseudo-time step and relaxation, marched from a seeded developed state
    of that cavity (the oracle cannot afford the GPU arm's spin-up from rest: one 101^3 step takes
    about 3.5 s on the machine's host cores). W warm-up steps, then K timed steps (at most 30, so that
    the run ends within a few minutes)."""
    from paper_2411_06563_gb300 import replicas as R
    ws, rank, _ = R.world()
    if rank != 0:
        return 0
    from oracle import hosc_oracle as O
    from paper_2411_06563_gb300 import inputs
    N = wl["N"]
    prm = O.Params(N=N, Ra=wl["Ra"], Pr=wl["Pr"], n=wl["n"], dt=wl["dt"], lam=wl["lam"],
                   tol_div=wl["tol_div"], tol_lin=1e-10, use_history=wl["history"])
    g = O.Grid(N)
    st = dict(inputs.cavity_state(N, wl["Ra"], seed=2411), prev=None, steps=0)
    for _ in range(args.warmup):
        st, _ = O.step(st, prm, g)
    k = max(1, min(args.steps, 30))
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(k):
        st, _ = O.step(st, prm, g)
    dt = time.perf_counter() - t0
    cores = _cores_used(time.process_time() - c0, dt)
    val = (N - 2) ** 3 * k / dt
    sample = "%d oracle steps of the %d^3 workload from a seeded developed state" % (k, N)
    out = {"impl": "reference", "metric": "grid-point updates/s", "value": val, "unit": "GPUPS",
           "n_gpus": args.gpus, "steps": k, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / k, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["desc"], "N": N, "Ra": wl["Ra"], "n": wl["n"],
                      "Pr": wl["Pr"], "dt": wl["dt"], "lambda": wl["lam"], "sample": sample},
           "cpu_baseline": dict({"value": val, "unit": "GPUPS", "cores": cores, "kind": "oracle",
                                 "sample": sample}, **_host()),
           "e2e": {"value": val, "unit": "GPUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _one_at_a_time(H, S, cavs, precision, steps, warmup):
    """Plain single-cavity solves, one after the other: GPUPS over the set (each cavity warmed
    up, then `steps` steps timed; device-synchronised host clock)."""
    import torch
    tot_pts, tot_s = 0.0, 0.0
    for c in cavs:
        p = S.request_params(c["N"], c["Ra"], c["n"], c["Pr"], precision=precision)
        with H.Cavity(p) as cav:
            cav.step(warmup)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = cav.step(steps)
            torch.cuda.synchronize()
            tot_s += time.perf_counter() - t0
            tot_pts += (c["N"] - 2) ** 3 * info["steps"]
    return tot_pts / tot_s


def run_batch(args):
    print(json.dumps(batch_line(args)))
    return 0


def batch_line(args):
    """Batched configuration: 64 uneven cavities (N in {21, 31, 41, 61}, log-uniform Ra in
    [1e2, 1e5], n uniform in [0.75, 1.25], Pr = 1, seed 20241106) advancing together in a pool,
    one captured graph launch per round of G steps for all cavities, launch shapes autotuned per
    N. value = aggregate GPUPS over the timed rounds; compared with the same cavities solved one
    at a time (mixed and plain FP64, GPUPS over a fixed step count each)."""
    import torch
    from paper_2411_06563_gb300 import hosc as H, inputs, serve as S
    cavs = inputs.batch_mix()
    G = args.round_steps
    mode = {"graph": H.HOSC_POOL_GRAPH, "streams": H.HOSC_POOL_STREAMS,
            "persistent": H.HOSC_POOL_PERSISTENT}[args.pool_mode]
    budget = sum(H.hosc_workspace_bytes(S.request_params(c["N"], c["Ra"], c["n"], c["Pr"]))
                 for c in cavs) + (1 << 20)
    rounds = max(1, args.steps // G)
    warm_rounds = max(3, args.warmup)
    with S.Pool(budget, G, mode, True) as pool:
        slots = [pool.admit(S.request_params(c["N"], c["Ra"], c["n"], c["Pr"]),
                            (warm_rounds + rounds) * G + G) for c in cavs]
        assert None not in slots
        for _ in range(warm_rounds):   # captures, per-N autotuning, first rounds
            assert not pool.run(1)
        torch.cuda.synchronize()
        steps0 = [pool.result(s)["info"]["steps"] for s in slots]
        t0 = time.perf_counter()
        for _ in range(rounds):
            pool.run(1)   # a cavity that completes stays in the pool, idle
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        st1 = pool.stats()
        res = [pool.result(s)["info"] for s in slots]
    pts = sum((c["N"] - 2) ** 3 * (r["steps"] - s0) for c, r, s0 in zip(cavs, res, steps0))
    iters = sum(r["lin_iters"] for r in res)
    value = pts / el
    sub = cavs[:args.baseline_cavities]
    one_mixed = _one_at_a_time(H, S, sub, H.HOSC_MIXED, args.baseline_steps, 5)
    one_fp64 = _one_at_a_time(H, S, sub, H.HOSC_FP64, args.baseline_steps, 5)
    out = {"metric": "grid-point updates/s (batched)", "value": value, "unit": "GPUPS",
           "n_gpus": 1, "steps": rounds * G, "warmup": warm_rounds * G,
           "ms_per_step": 1e3 * el / (rounds * G), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "batch of 64 cavities, N in {21,31,41,61}, Ra log-uniform "
                                  "[1e2,1e5], n uniform [0.75,1.25], Pr=1, seed 20241106, mixed",
                      "pool_mode": args.pool_mode, "steps_per_round": G,
                      "graph_launches_timed": rounds if mode == H.HOSC_POOL_GRAPH else None,
                      "round_kernel_launches_timed":
                          rounds if mode == H.HOSC_POOL_PERSISTENT else None,
                      "captures": st1["captures"], "capture_ms": st1["capture_ms"],
                      "tuned_sizes": st1["tuned_sizes"],
                      "bicgstab_iters_per_cavity_step":
                          iters / (4.0 * max(1, sum(r["steps"] for r in res))),
                      "dt": "per cavity from the steady-solve rule (hosc_steady_params)"},
           "one_at_a_time": {"cavities": len(sub), "steps_each": args.baseline_steps,
                             "mixed_GPUPS": one_mixed, "fp64_GPUPS": one_fp64,
                             "batched_over_fp64": value / one_fp64,
                             "batched_over_mixed": value / one_mixed}}
    return out


def steady_solve(H, N, Ra, n, Pr=1.0, max_steps=200000, precision=None, stream=None,
                 max_seconds=1e9):
    """One steady solve with the library's steady-solve parameters (hosc_steady_params), mixed
    precision with the automatic switch to FP64 defect sweeps, from rest to max|chi^{n+1} -
    chi^n|/dt < 1e-6 and max|div V| < 1e-6. Returns a dict: wall seconds (device-synchronised),
    steps, iterations, status, diagnostics and a summary of the local entropy field."""
    import numpy as np
    import torch
    p = H.hosc_steady_params(N, Ra, Pr, n)
    p.precision = H.HOSC_MIXED if precision is None else precision
    p.tol_lin = 1e-10
    if stream is not None:
        p.cuda_stream = stream.cuda_stream
    with H.Cavity(p) as cav:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done, info, switch, chunk, lin = 0, None, None, 1000, 0
        while done < max_steps:   # chunks, with progress on stderr
            info = cav.solve_steady(min(chunk, max_steps - done),
                                    allow=(H.HOSC_ESTEPLIMIT, H.HOSC_ENOCONV, H.HOSC_EDIVERGED))
            done += info["steps"]
            lin += info["lin_iters"]
            phase = H.hosc_get_phase(cav.h)
            if phase == 1 and switch is None:
                switch = done   # the automatic switch happened within this chunk
            last = info["call_status"] != H.HOSC_ESTEPLIMIT or \
                time.perf_counter() - t0 > max_seconds
            if done % (5 * chunk) == 0 or last:
                print("steady %d^3: %d steps, res/dt %.3e, div %.3e, phase %d, %.0f s" % (
                    N, done, info["res"] / p.dt, info["div_max"], phase,
                    time.perf_counter() - t0), file=sys.stderr, flush=True)
            if last:
                break
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        info["steps"] = done
        d = cav.diagnostics(with_fields=True)
        phase = H.hosc_get_phase(cav.h)
    el_f = d["E_local_field"]
    z = d["Nu_avg_z"]
    peaks = int(np.sum((z[1:-1] > z[:-2]) & (z[1:-1] > z[2:])))
    return {"N": N, "Ra": Ra, "n": n, "Pr": Pr, "dt": p.dt, "lambda": p.lambda_,
            "status": H.hosc_strerror(info["call_status"]), "steady": info["call_status"] == 0,
            "steps": info["steps"], "seconds": el,
            "GPUPS": (N - 2) ** 3 * info["steps"] / el if el > 0 else None,
            "bicgstab_iters_per_step": lin / (4.0 * max(1, done)),
            "res_over_dt": info["res"] / p.dt, "div_max": info["div_max"],
            "stop": {"tol_steady": p.tol_steady, "div_steady": p.div_steady,
                     "tol_div_correction": p.tol_div},
            "final_phase": "FP64 defect sweeps" if phase == 1 else "FP32 sweeps",
            "defect_switch_by_step": switch,
            "Nu_mean": d["Nu_hot_mean"], "Nu_max": d["Nu_hot_max"],
            "Nu_cold_mean": d["Nu_cold_mean"], "E_total": d["E_total"], "E_HT": d["E_HT"],
            "E_FF": d["E_FF"], "Be": d["Be"], "Nu_avg_z_local_maxima": peaks,
            "E_local_field": {"min": float(el_f.min()), "max": float(el_f.max()),
                              "mean": float(el_f.mean())}}


def run_steady(args):
    """Steady solve of the single large cavity (101^3, n = 0.75, Ra = 1e5, Pr = 1, mixed
    precision with FP64 defect sweeps) from rest: solves/s, steps, Nu, Be and the local entropy
    generation field."""
    import torch
    from paper_2411_06563_gb300 import hosc as H
    torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    r = steady_solve(H, wl["N"], wl["Ra"], wl["n"], wl["Pr"], args.max_steps,
                     max_seconds=args.max_seconds)
    out = {"metric": "steady solves/s", "value": 1.0 / r["seconds"], "unit": "solves/s",
           "n_gpus": 1, "steps": r["steps"], "warmup": 0,
           "ms_per_step": 1e3 * r["seconds"] / max(1, r["steps"]),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic", "config": {"workload": wl["desc"]},
           "steady": r}
    print(json.dumps(out))
    return 0


def run_table1(args):
    """The grid study of Table 1 (Sec. 3.1): n = 0.75, Ra = 1e4, Pr = 1, the three-level scheme,
    marched from rest to t = 100 on each requested grid (dt = 5e-4, inside the stability bound of
    the printed scheme at this Ra; mixed precision with FP64 defect sweeps once the step change
    stalls), with theta, u, v, w at the probes (0.6, 0.6, 0.6) and (0.4, 0.4, 0.4) beside the
    printed values. The steady state is centro-symmetric here (theta_ref = 1/2), so the printed
    (0.6, 0.6, 0.6) values are also set beside this march's (0.4, 0.4, 0.4) ones."""
    import torch
    from paper_2411_06563_gb300 import hosc as H
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from golden_values import table
    from test_gpu_table1 import table1_params
    torch.cuda.set_device(0)
    printed = {(r[0], int(r[3])): r[4:] for r in table("table1_probes.txt")}
    out = []
    for N in (int(x) for x in args.table1_sizes.split(",")):
        p = table1_params(N, H.HOSC_MIXED)
        p.tol_lin = 1e-10
        steps = int(round(100.0 / p.dt))
        with H.Cavity(p) as cav:
            t0 = time.perf_counter()
            done = 0
            while done < steps:
                info = cav.step(min(5000, steps - done))
                done += info["steps"]
                if info["call_status"] not in (0,):
                    break
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            f = {k: cav.get(w) for k, w in (("th", H.HOSC_THETA), ("u", H.HOSC_U),
                                           ("v", H.HOSC_V), ("w", H.HOSC_W))}
            phase = H.hosc_get_phase(cav.h)
        probes = {}
        for x in (0.6, 0.4):
            i = int(round(x * (N - 1)))
            probes[str(x)] = [float(f[k][i, i, i]) for k in ("th", "u", "v", "w")]
        row = {"N": N, "dt": p.dt, "lambda": p.lambda_, "steps": done, "t": done * p.dt,
               "status": H.hosc_strerror(info["call_status"]), "seconds": el,
               "res_over_dt_last": info["res"] / p.dt, "div_max_last": info["div_max"],
               "final_phase": "FP64 defect sweeps" if phase == 1 else "FP32 sweeps",
               "probes_theta_u_v_w": probes,
               "printed": {str(x): list(printed.get((x, N), [])) for x in (0.6, 0.4)}}
        out.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    res = {"metric": "Table 1 march to t = 100", "value": None, "unit": "probe values",
           "n_gpus": 1, "data": "synthetic", "table1": out}
    print(json.dumps(res))
    return 0


def run_equal(args):
    """Steady solves at equal accuracy: a seeded set of small cavities (N in {17, 21}, Ra
    log-uniform in [1e2, 1e3], n uniform in [0.9, 1.1], Pr = 1, dt = 0.02, lambda = 0.1,
    tol_steady = tol_div = 1e-6), each solved to steady state by the plain FP64 path one at a
    time, then all together in a mixed-precision pool (FP32 sweeps, FP64 defect sweeps once the
    step change stalls). value = pool solves/s; the line carries the FP64 solves/s and the
    largest field and Nu differences between the two."""
    import numpy as np
    import torch
    from paper_2411_06563_gb300 import hosc as H, inputs, serve as S
    c4 = args.equal_mix == "c4"
    cavs = (inputs.batch_mix()[:args.equal_cavities] if c4
            else inputs.steady_mix(args.equal_cavities))
    fields = (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W), ("th", H.HOSC_THETA))

    def params(c, precision):
        if c4:   # the steady-solve rule, tol_steady = 1e-6
            return S.request_params(c["N"], c["Ra"], c["n"], c["Pr"], precision=precision)
        p = S.request_params(c["N"], c["Ra"], c["n"], c["Pr"], precision=precision,
                             tol_steady=1e-6, tol_div=1e-6)
        p.dt = 0.02
        p.lambda_ = 0.1
        return p

    ref = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in cavs:
        with H.Cavity(params(c, H.HOSC_FP64)) as cav:
            info = cav.solve_steady(args.equal_max_steps)
            ref.append(dict(info=info, diag=cav.diagnostics(),
                            **{k: cav.get(w) for k, w in fields}))
            print("fp64 %s: %d steps, %s, %.0f s" % (c, info["steps"], info["call_status"],
                                                     time.perf_counter() - t0),
                  file=sys.stderr, flush=True)
    t64 = time.perf_counter() - t0
    budget = sum(H.hosc_workspace_bytes(params(c, H.HOSC_MIXED)) for c in cavs) + (1 << 20)
    mode = {"graph": H.HOSC_POOL_GRAPH, "streams": H.HOSC_POOL_STREAMS,
            "persistent": H.HOSC_POOL_PERSISTENT}[args.pool_mode]
    got = {}
    t0 = time.perf_counter()
    with S.Pool(budget, args.round_steps, mode, True) as pool:
        slots = [pool.admit(params(c, H.HOSC_MIXED), args.equal_max_steps) for c in cavs]
        while len(got) < len(cavs):
            for s_ in pool.run(64):
                got[s_] = pool.result(s_, fields)
        tmx = time.perf_counter() - t0
        pst = pool.stats()
    mix = [got[s_] for s_ in slots]
    steady64 = sum(1 for r in ref if r["info"]["call_status"] == 0)
    steadymx = sum(1 for r in mix if r["status"] == 0)
    dfield = max(float(np.max(np.abs(a[k] - b[k]))) for a, b in zip(mix, ref) for k, _ in fields)
    dnu = max(abs(a["diag"]["Nu_hot_mean"] - b["diag"]["Nu_hot_mean"]) / abs(b["diag"]["Nu_hot_mean"])
              for a, b in zip(mix, ref))
    out = {"metric": "steady cavity solves/s at equal accuracy", "value": len(cavs) / tmx,
           "unit": "solves/s", "n_gpus": 1, "steps": len(cavs), "warmup": 0,
           "ms_per_step": 1e3 * tmx / len(cavs), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": ("the first %d cavities of the 64-cavity mix (N in "
                                   "{21,31,41,61}, Ra log-uniform [1e2,1e5], n uniform "
                                   "[0.75,1.25], seed 20241106), steady-solve rule, "
                                   "tol_steady=1e-6" % len(cavs)) if c4 else
                                  ("%d cavities N in {17,21}, Ra log-uniform [1e2,1e3], n uniform "
                                   "[0.9,1.1], Pr=1, dt=0.02, lambda=0.1, tol_steady=tol_div=1e-6, "
                                   "seed 20241108" % len(cavs)),
                      "pool_mode": args.pool_mode, "steps_per_round": args.round_steps,
                      "captures": pst["captures"]},
           "fp64_one_at_a_time": {"solves_per_s": len(cavs) / t64, "seconds": t64,
                                  "steady": steady64,
                                  "steps": [r["info"]["steps"] for r in ref]},
           "mixed_pool": {"seconds": tmx, "steady": steadymx,
                          "steps": [r["info"]["steps"] for r in mix]},
           "speedup_over_fp64": t64 / tmx,
           "accuracy": {"max_abs_field_diff": dfield, "max_rel_Nu_diff": dnu,
                        "targets": {"field": 1e-5, "Nu": 1e-4}}}
    print(json.dumps(out))
    return 0


def run_serve(args):
    print(json.dumps(serve_line(args, newtonian_only=args.newtonian_only)))
    return 0


def serve_line(args, saturated_only=False, newtonian_only=False):
    """Serving configuration: a seeded Poisson stream (seed 20241107) of cavity solves, N in
    {21, 31, ..., 101}, log-uniform Ra in [1e2, 1e5], n in {0.75, 1.0, 1.25}, Pr = 1, admitted
    against a device-memory budget, each solved to steady state (max|chi^{n+1} - chi^n|/dt and
    max|div V| below tol_steady, 1e-6) with the library's steady-solve rule, or to a step cap, in
    a pool. The first `saturation_requests` requests all present at t = 0 give the saturated
    rate; then (unless saturated_only) the first `requests` requests of the stream arrive at rho
    times that rate. newtonian_only keeps the stream's n = 1 requests, in their order (the
    power-law requests at low Ra need 10^5 steps and more to reach the stop). Solves/s and p50 /
    p99 arrival-to-completion times."""
    from paper_2411_06563_gb300 import hosc as H, inputs, serve as S
    mode = {"graph": H.HOSC_POOL_GRAPH, "streams": H.HOSC_POOL_STREAMS,
            "persistent": H.HOSC_POOL_PERSISTENT}[args.pool_mode]
    budget = int(args.budget_gb * (1 << 30))

    def make(r):
        return S.request_params(r["N"], r["Ra"], r["n"], r["Pr"], tol_steady=args.tol_steady)

    max_steps = args.max_steps
    # a prefix of the configured stream of 2000 requests (the parameters of request q do not
    # depend on the rate, only its arrival time does)
    total = max(args.requests, args.saturation_requests, 2000)
    keep = (lambda r: r["n"] == 1.0) if newtonian_only else (lambda r: True)
    base = [r for r in inputs.request_stream(total, rate=1.0) if keep(r)]
    sat_reqs = [dict(r, t=0.0) for r in base[:args.saturation_requests]]
    with S.Pool(budget, args.round_steps, mode, True) as pool:
        sres, sat = S.serve(sat_reqs, pool, make, max_steps)
        pst = pool.stats()
    if saturated_only:
        res, summ, n_req, rho = sres, sat, len(sat_reqs), None
    else:
        rate = args.rho * sat["solves_per_s"]
        stream = [r for r in inputs.request_stream(total, rate=rate) if keep(r)][:args.requests]
        with S.Pool(budget, args.round_steps, mode, True) as pool:
            res, summ = S.serve(stream, pool, make, max_steps)
            pst = pool.stats()
        n_req, rho = args.requests, args.rho
    out = {"metric": "served cavity solves/s", "value": summ["solves_per_s"], "unit": "solves/s",
           "n_gpus": 1, "steps": n_req, "warmup": 0,
           "ms_per_step": 1e3 / summ["solves_per_s"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "p50_s": summ["p50_s"], "p99_s": summ["p99_s"],
           "seed_prefix": "the first %d %srequests of the seeded stream (arrival order)%s"
                          % (n_req, "Newtonian (n = 1) " if newtonian_only else "",
                             ", all present at t = 0" if saturated_only else ""),
           "config": {"workload": "Poisson stream of cavity solves, N in {21..101} step 10, Ra "
                                  "log-uniform [1e2,1e5], n in {0.75,1,1.25}, Pr=1, seed "
                                  "20241107, the library's steady-solve rule",
                      "rho": rho, "saturated_solves_per_s": sat["solves_per_s"],
                      "saturation_requests": len(sat_reqs), "budget_GB": args.budget_gb,
                      "max_steps": max_steps, "tol_steady": args.tol_steady,
                      "pool_mode": args.pool_mode, "steps_per_round": args.round_steps,
                      "completed": summ["completed"], "steady": summ["steady"],
                      "requests": [{k: r[k] for k in ("N", "Ra", "n")}
                                   for r in base[:n_req]],
                      "steps_to_steady": [r.get("steps") if r else None for r in res],
                      "latency_s": [r.get("latency") if r else None for r in res],
                      "captures": pst["captures"], "capture_ms": pst["capture_ms"]}}
    return out


def _pool_blocks(args):
    """Bounded runs of the batching and serving workloads for the default line: the 64-cavity
    mix advanced 32 steps in rounds of 8 (after 3 warm-up rounds) against 4 of its cavities one
    at a time, and the first `serve_block_requests` Newtonian requests of the serving stream, all
    present at t = 0, each solved to steady state."""
    import types
    common = dict(pool_mode="graph", round_steps=8, budget_gb=64.0)
    t0 = time.perf_counter()
    b = batch_line(types.SimpleNamespace(steps=32, warmup=3, baseline_cavities=4,
                                         baseline_steps=20, **common))
    t1 = time.perf_counter()
    s = serve_line(types.SimpleNamespace(requests=args.serve_block_requests,
                                         saturation_requests=args.serve_block_requests,
                                         rho=None, max_steps=300000, tol_steady=1e-6,
                                         **common), saturated_only=True, newtonian_only=True)
    t2 = time.perf_counter()
    keep = ("metric", "value", "unit", "steps", "ms_per_step")
    batch = dict({k: b[k] for k in keep}, config=b["config"], one_at_a_time=b["one_at_a_time"],
                 wall_s=t1 - t0)
    serve = dict({k: s[k] for k in keep}, p50_s=s["p50_s"], p99_s=s["p99_s"],
                 seed_prefix=s["seed_prefix"], config=s["config"], wall_s=t2 - t1)
    return {"batch": batch, "serve": serve}


def _host():
    """Host CPU model and logical CPU count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        if model:
            raise OSError
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"host_cpus": os.cpu_count(), "cpu_model": model}


_ONE_THREAD_STEP = r"""
import sys, time, numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import hosc_oracle as O
z = np.load(sys.argv[2], allow_pickle=False)
prm = O.Params(N=int(z["N"]), Ra=float(z["Ra"]), Pr=float(z["Pr"]), n=float(z["n"]),
               dt=float(z["dt"]), lam=float(z["lam"]), tol_lin=float(z["tol"]),
               use_history=int(z["hist"]))
prev = None
if int(z["hist"]):
    prev = {k: z["prev_" + k] for k in ("L", "u", "v", "w", "Eu", "Ev", "Ew")}
st = dict(u=z["u"], v=z["v"], w=z["w"], th=z["th"], p=z["p"], steps=0, prev=prev)
g = O.Grid(prm.N)
k = int(sys.argv[3]) if len(sys.argv) > 3 else 1
t0 = time.perf_counter()
for _ in range(k):
    st, _info = O.step(st, prm, g)
print((time.perf_counter() - t0) / k)
"""


def _one_thread_step(st, prm, path, steps=1):
    """Wall time per oracle step (mean over `steps` steps from the same state) in a child process
    held to one thread (OMP, OpenBLAS and MKL thread pools of numpy and scipy set to 1)."""
    arrays = {k: st[k] for k in ("u", "v", "w", "th", "p")}
    hist = st.get("prev") is not None
    if hist:
        arrays.update({"prev_" + k: v for k, v in st["prev"].items()})
    import numpy as np
    np.savez(path, N=prm.N, Ra=prm.Ra, Pr=prm.Pr, n=prm.n, dt=prm.dt, lam=prm.lam,
             tol=prm.tol_lin, hist=int(hist), **arrays)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", _ONE_THREAD_STEP, ROOT, path, str(steps)],
                         env=env, capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        return None
    return float(out.stdout.strip().splitlines()[-1])


def _cores_used(cpu_s, wall_s):
    """Threads the oracle kept busy over a timed interval: process CPU time over wall time (the
    oracle itself is single-threaded; numpy's BLAS may add threads for long vectors)."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


def cpu_baseline(cav, H, wl):
    """One oracle step of the same 101^3 workload from the GPU's current state (with history)."""
    import numpy as np
    from oracle import hosc_oracle as O
    N = wl["N"]
    prm = O.Params(N=N, Ra=wl["Ra"], Pr=wl["Pr"], n=wl["n"], dt=wl["dt"],
                   lam=cav.params.lambda_, tol_lin=cav.params.tol_lin,
                   tol_div=cav.params.tol_div, use_history=wl["history"])
    st = dict(u=cav.get(H.HOSC_U), v=cav.get(H.HOSC_V), w=cav.get(H.HOSC_W),
              th=cav.get(H.HOSC_THETA), p=cav.get(H.HOSC_P), steps=0,
              prev=dict(L=cav.get(H.HOSC_PREV_L), u=cav.get(H.HOSC_PREV_U),
                        v=cav.get(H.HOSC_PREV_V), w=cav.get(H.HOSC_PREV_W),
                        Eu=cav.get(H.HOSC_PREV_EU), Ev=cav.get(H.HOSC_PREV_EV),
                        Ew=cav.get(H.HOSC_PREV_EW)))
    g = O.Grid(N)
    t0, c0 = time.perf_counter(), time.process_time()
    O.step(st, prm, g)
    dt = time.perf_counter() - t0
    cores = _cores_used(time.process_time() - c0, dt)
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        dt1 = _one_thread_step(st, prm, path)
    finally:
        os.unlink(path)
    out = {"value": (N - 2) ** 3 / dt, "unit": "GPUPS", "cores": cores, "kind": "oracle",
           "sample": "1 oracle step of the %d^3 workload from the GPU state (%.1f s)" % (N, dt),
           "one_thread": ({"value": (N - 2) ** 3 / dt1, "unit": "GPUPS", "cores": 1,
                           "seconds": dt1} if dt1 else None),
           "by_config": _oracle_config_timings(H)}
    out.update(_host())
    return out


def _oracle_config_timings(H, steps=3):
    """The oracle on the other single-cavity configurations: the Newtonian 21^3 cavity (Ra = 1e3)
    and the 41^3 power-law cavities (Ra = 1e4, n = 0.75 and 1.25), each from a seeded developed
    state at the steady-solve rule's step, `steps` steps with numpy's threads and on one thread."""
    from oracle import hosc_oracle as O
    from paper_2411_06563_gb300 import inputs
    rows = {}
    for name, N, Ra, n in (("C1 21^3 n=1 Ra=1e3", 21, 1e3, 1.0),
                           ("C2 41^3 n=0.75 Ra=1e4", 41, 1e4, 0.75),
                           ("C2 41^3 n=1.25 Ra=1e4", 41, 1e4, 1.25)):
        p = H.hosc_steady_params(N, Ra, 1.0, n)
        prm = O.Params(N=N, Ra=Ra, Pr=1.0, n=n, dt=p.dt, lam=p.lambda_, tol_lin=1e-12,
                       tol_div=p.tol_div, use_history=0)
        st = dict(inputs.cavity_state(N, Ra, seed=2024), steps=0, prev=None)
        g = O.Grid(N)
        s0, c0 = time.perf_counter(), time.process_time()
        cur = st
        for _ in range(steps):
            cur, _ = O.step(cur, prm, g)
        wall = (time.perf_counter() - s0) / steps
        cores = _cores_used(time.process_time() - c0, wall * steps)
        fd, path = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        try:
            one = _one_thread_step(st, prm, path, steps)
        finally:
            os.unlink(path)
        rows[name] = {"GPUPS": (N - 2) ** 3 / wall, "cores": cores,
                      "one_thread_GPUPS": (N - 2) ** 3 / one if one else None,
                      "steps": steps}
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity101", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the timing of the solver variant outside the paper's method")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape of the mixed-precision solve")
    ap.add_argument("--tiles", default=None,
                    help="launch shape of the mixed-precision solve as BLOCK,KZ,NARROW "
                         "(instead of the autotuner)")
    ap.add_argument("--tma-tiles", default=None,
                    help="bulk-copy stencil kernels as ROWS,PLANES,STAGES,KERNELS (with --tiles; "
                         "KERNELS 1 p/v, 2 s/t, 3 both)")
    ap.add_argument("--xr-form", type=int, default=None, choices=[0, 1],
                    help="x/r kernel: 0 column march, 1 flat stream (with --tiles)")
    ap.add_argument("--spinup", type=int, default=None,
                    help="untimed steps from rest before the warm-up (default: per workload)")
    ap.add_argument("--mode", default="step",
                    choices=["step", "batch", "serve", "equal", "steady", "table1"],
                    help="step: the single-cavity headline; batch: 64 cavities in a pool; "
                         "serve: a Poisson request stream on a pool; equal: steady solves of "
                         "the pool against one-at-a-time FP64 at equal accuracy")
    ap.add_argument("--equal-cavities", type=int, default=8)
    ap.add_argument("--equal-mix", default="c4", choices=["c4", "small"],
                    help="equal mode: the head of the 64-cavity mix, or the small steady mix")
    ap.add_argument("--table1-sizes", default="11,51")
    ap.add_argument("--max-seconds", type=float, default=1e9,
                    help="steady mode: stop after this wall time (status: step limit)")
    ap.add_argument("--equal-max-steps", type=int, default=20000)
    ap.add_argument("--pool-mode", default="graph",
                    choices=["graph", "streams", "persistent"])
    ap.add_argument("--round-steps", type=int, default=8)
    ap.add_argument("--baseline-cavities", type=int, default=16)
    ap.add_argument("--baseline-steps", type=int, default=40)
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--saturation-requests", type=int, default=32)
    ap.add_argument("--rho", type=float, default=0.8)
    ap.add_argument("--no-pool-blocks", action="store_true",
                    help="leave the bounded batch and serve blocks out of the default line")
    ap.add_argument("--serve-block-requests", type=int, default=6)
    ap.add_argument("--newtonian-only", action="store_true",
                    help="serve mode: keep the stream's n = 1 requests")
    ap.add_argument("--max-steps", type=int, default=1000)
    ap.add_argument("--tol-steady", type=float, default=1e-6)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "ours" and args.mode == "batch":
        return run_batch(args)
    if args.impl == "ours" and args.mode == "serve":
        return run_serve(args)
    if args.impl == "ours" and args.mode == "equal":
        return run_equal(args)
    if args.impl == "ours" and args.mode == "steady":
        return run_steady(args)
    if args.impl == "ours" and args.mode == "table1":
        return run_table1(args)
    if args.impl == "reference":
        return run_reference(args, wl)

    import numpy as np
    import torch
    from paper_2411_06563_gb300 import replicas as R
    ws, rank, local = R.world()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2411_06563_gb300 import hosc as H

    N = wl["N"]
    h = 1.0 / (N - 1)
    stream = torch.cuda.current_stream()
    spinup = wl["spinup"] if args.spinup is None else args.spinup

    def make(precision, precond=0, solver=0):
        p = H.hosc_steady_params(N, wl["Ra"], wl["Pr"], wl["n"])
        assert (p.dt, p.lambda_, p.tol_div) == (wl["dt"], wl["lam"], wl["tol_div"]), \
            "the workload table no longer matches the library's steady-solve rule"
        p.precond = precond
        p.solver = solver
        p.tol_lin = 1e-10
        p.use_history = wl["history"]
        p.precision = H.HOSC_MIXED if precision == "mixed" else H.HOSC_FP64
        p.auto_defect = 0   # time the FP32 sweeps; the FP64 defect phase is for the last digits
        p.cuda_stream = stream.cuda_stream
        cav = H.Cavity(p, workspace="torch")
        # spin-up from rest (untimed), then the launch-shape autotuner (mixed precision), then
        # warm-up steps
        info = cav.step(spinup)
        assert info["call_status"] == 0, info
        if precision == "mixed" and args.tiles:
            kb, kz, nr = (int(x) for x in args.tiles.split(","))
            rc = H.hosc_set_tiles(cav.h, kb, kz, nr)
            assert rc == 0, ("launch shape", args.tiles, rc)
            if args.tma_tiles:
                ty, tz, ts, tk = (int(x) for x in args.tma_tiles.split(","))
                rc = H.hosc_set_tma_tiles(cav.h, ty, tz, ts, tk)
                assert rc == 0, ("bulk-copy shape", args.tma_tiles, rc)
            if args.xr_form is not None:
                assert H.hosc_set_xr_form(cav.h, args.xr_form) == 0
        elif precision == "mixed" and not args.no_autotune:
            rc, kb, kz, _ = H.hosc_autotune(cav.h, 5)
            assert rc == 0, rc
        cav.step(args.warmup)
        torch.cuda.synchronize()
        return p, cav

    barrier = R.barrier

    fp64_compare = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        # the plain all-FP64 path on the same workload, for context, with BiCGSTAB and with
        # BiCGSTAB(2) (the two readings of the paper's solver): iterations x bytes per step
        fp64_compare = {}
        for name, solver in (("bicgstab", 0), ("bicgstab2", 1)):
            p64, c64 = make("fp64", solver=solver)
            k64 = max(5, args.steps // 4)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            ea.record(stream)
            i64 = c64.step(k64)
            eb.record(stream)
            torch.cuda.synchronize()
            fp64_compare[name] = {
                "value": (N - 2) ** 3 * k64 * ws / (ea.elapsed_time(eb) * 1e-3),
                "steps": k64, "ms_per_step": ea.elapsed_time(eb) / k64,
                # iterations: operator-application pairs per system and step (a BiCGSTAB(2)
                # cycle counts two)
                "iters_per_step": i64["lin_iters"] / (4.0 * i64["steps"]),
                # algorithmic bytes per iteration and interior node, four systems: BiCGSTAB
                # 96 words (p/v 38, s/t 26, x/r 32); BiCGSTAB(2) 224 words per two-iteration
                # cycle (B1 30, B2 50, B3 46, B4 54, B5 44)
                "krylov_bytes_per_iteration_per_node": 768 if solver == 0 else 896}
            if solver == 0:
                fp64_compare[name]["roofline"] = _fp64_roofline(H, c64, N)
            c64.close()
    p, cav = make(args.precision)

    # ------------------------------------------------------------- timed region (device-resident)
    l0 = cav.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        info = cav.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
    ms = e0.elapsed_time(e1)
    launches = cav.kernel_launches() - l0
    ms = R.max_over_ranks(ms)   # replicas: each rank ran its own cavity
    units = (N - 2) ** 3 * args.steps * ws
    value = units / (ms * 1e-3)
    lin_iters = info["lin_iters"]

    # ------------------------------------------------------------- kernel breakdown (events)
    H.hosc_profile_enable(cav.h, 1)
    prof_steps = max(5, min(args.steps, 50))
    torch.cuda.nvtx.range_push("profiled_steps")   # uncaptured steps: one launch per kernel
    cav.step(prof_steps)
    torch.cuda.nvtx.range_pop()
    names = ["k_viscosity", "k_sources", "k_rhs", "k_bicg_pv", "k_bicg_st", "k_bicg_xr", "update"]
    kern = {}
    for kid, name in enumerate(names):
        _, kms, kl, kb = H.hosc_profile_read(cav.h, kid)
        kern[name] = dict(ms=kms, launches=kl, bytes=kb)
    H.hosc_profile_enable(cav.h, 0)
    # each class alone, launched back to back on the current buffers (no host gaps), inside an
    # NVTX range that a profiler can select
    iso = {}
    torch.cuda.nvtx.range_push("kernels_alone")
    for kid, name in enumerate(names[:6]):
        rc, kms, kb = H.hosc_time_kernel(cav.h, kid, 20)
        if rc == 0:
            iso[name] = {"us_per_launch": kms * 1e3,
                         "GBps": kb / (kms * 1e-3) / 1e9 if kb > 0 and kms > 0 else 0.0}
    torch.cuda.nvtx.range_pop()
    dom = max(kern, key=lambda k: kern[k]["ms"])
    peak, peak_kind = _peaks()
    d = kern[dom]
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    total_ms = sum(k["ms"] for k in kern.values())

    # ------------------------------------------------------------- end to end through host buffers
    e2e_steps = max(3, min(args.steps // 10, 20))
    n3 = N ** 3
    which = [H.HOSC_U, H.HOSC_V, H.HOSC_W, H.HOSC_THETA, H.HOSC_P]
    host = [torch.empty((N, N, N), dtype=torch.float64, pin_memory=True).numpy() for _ in which]
    for a, w_ in zip(host, which):
        H.hosc_get_field(cav.h, w_, a)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for a, w_ in zip(host, which):
            H.hosc_set_field(cav.h, w_, a)
        H.hosc_step(cav.h, 1)
        for a, w_ in zip(host, which):
            H.hosc_get_field(cav.h, w_, a)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = R.max_over_ranks(e2e_s)
    e2e_val = (N - 2) ** 3 * e2e_steps * ws / e2e_s

    mixed = args.precision == "mixed"
    shape = {"tiles": dict(zip(("block", "kz", "narrow"), H.hosc_get_tiles(cav.h)[1:]))
             if mixed else None,
             "stencil": dict(zip(("sx", "sy", "skz"), H.hosc_get_stencil_tiles(cav.h)[1:]))
             if mixed else None,
             "tma": dict(zip(("rows", "planes", "stages", "kernels"),
                             H.hosc_get_tma_tiles(cav.h)[1:]))
             if mixed else None,
             "xr": (("flat stream" if H.hosc_get_xr_form(cav.h) else "column march")
                    if mixed else None),
             "form": (("merged: 2 kernels per iteration" if H.hosc_get_krylov_merged(cav.h)
                       else "3 kernels per iteration") if mixed else None)}
    traffic = None
    if mixed:
        traffic = NCU_TRAFFIC.get((args.workload, dom, _kernel_shape(dom, shape)))
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cav, H, wl)
    pool_blocks = None
    if rank == 0 and ws == 1 and args.precision == "mixed" and not args.no_pool_blocks:
        pool_blocks = _pool_blocks(args)

    # a variant outside the paper's method, for comparison only: the same workload with Jacobi
    # row scaling of the level-(n+1) systems before BiCGSTAB (same solution, fewer iterations)
    variant = None
    if args.precision == "mixed" and not args.no_variants:
        cav.close()
        pj, cj = make("mixed", precond=1)
        kj = max(20, args.steps // 2)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ea.record(stream)
        ij = cj.step(kj)
        eb.record(stream)
        torch.cuda.synchronize()
        msj = R.max_over_ranks(ea.elapsed_time(eb))
        variant = {"jacobi_row_scaling": {
            "value": (N - 2) ** 3 * kj * ws / (msj * 1e-3), "unit": "GPUPS", "steps": kj,
            "ms_per_step": msj / kj,
            "bicgstab_iters_per_step": ij["lin_iters"] / (4.0 * kj),
            "note": "not the paper's solver: each row of the level-(n+1) systems scaled by its "
                    "diagonal before the unpreconditioned BiCGSTAB"}}
        cav = cj

    if rank == 0:
        out = {
            "metric": "grid-point updates/s", "value": value, "unit": "GPUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "N": N, "Ra": wl["Ra"], "n": wl["n"],
                       "Pr": wl["Pr"], "dt": wl["dt"], "precision": args.precision,
                       "mixed_phase": "FP32 sweeps and Krylov, FP64 state/reductions/pressure"
                       if args.precision == "mixed" else None,
                       "fp64_path": fp64_compare,
                       "spinup_steps": spinup, "tol_lin": p.tol_lin,
                       "use_history": wl["history"], "lambda": p.lambda_,
                       "bicgstab_iters_per_step": lin_iters / (4.0 * args.steps),
                       # per system (u, v, w, theta), and the passes of the interleaved solve
                       # (it iterates the four systems together until the last has converged)
                       "iters_per_step_by_system": dict(zip(
                           ("u", "v", "w", "theta"),
                           (x / args.steps for x in info["sys_iters"]))),
                       "solve_passes_per_step": info["solve_iters"] / args.steps,
                       "lane_utilisation": (lin_iters / (4.0 * info["solve_iters"])
                                            if info["solve_iters"] else None),
                       # interior nodes x systems x BiCGSTAB iterations per second
                       "sweep_rate_per_s": (N - 2) ** 3 * lin_iters * ws / (ms * 1e-3),
                       "krylov_tiles": shape["tiles"], "stencil_tiles": shape["stencil"],
                       "tma_tiles": shape["tma"], "xr_form": shape["xr"],
                       "krylov_form": shape["form"],
                       "l2": "no flush: device working set %.0f MB > 129 MB L2"
                             % (H.hosc_workspace_bytes(p) / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "share": d["ms"] / total_ms if total_ms else None},
            "kernels_alone": iso,
            "kernels": {k: {"ms_per_step": v["ms"] / prof_steps, "launches": v["launches"],
                            "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] else 0.0}
                        for k, v in kern.items()},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_val, "unit": "GPUPS", "h2d_bytes_per_step": 5 * n3 * 8,
                    "d2h_bytes_per_step": 5 * n3 * 8 + 64},
            "cpu_baseline": cpu,
            "variants": variant,
        }
        if pool_blocks:
            out.update(pool_blocks)
        print(json.dumps(out))
    cav.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
