"""Host-side checks of the benchmark's tables (no GPU): the workload table follows the library's
steady-solve rule, and every recorded DRAM-traffic entry is keyed by a launch shape that the
benchmark can report."""

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_workloads_follow_the_steady_rule():
    """The pseudo-time step, relaxation and correction threshold of each benchmark workload are
    those hosc_steady_params gives (the benchmark asserts the same at run time)."""
    H = pytest.importorskip("paper_2411_06563_gb300.hosc")
    B = _bench()
    for name, wl in B.WORKLOADS.items():
        p = H.hosc_steady_params(wl["N"], wl["Ra"], wl["Pr"], wl["n"])
        assert (p.dt, p.lambda_, p.tol_div) == (wl["dt"], wl["lam"], wl["tol_div"]), name
        assert p.div_steady == p.tol_steady == 1e-6


def test_traffic_table_keys_are_reportable_shapes():
    """Each NCU_TRAFFIC key names a known workload, a Krylov kernel class and a launch shape in the
    form _kernel_shape returns for that class; the traffic values are positive and below twice
    the class's algorithmic bytes (no entry can hide a re-read problem behind a typo)."""
    B = _bench()
    per_node = {"k_bicg_pv": 132, "k_bicg_st": 84, "k_bicg_xr": 128}
    for (wl, kernel, shape), traffic in B.NCU_TRAFFIC.items():
        assert wl in B.WORKLOADS and kernel in per_node
        N = B.WORKLOADS[wl]["N"]
        assert 0 < traffic < 2 * per_node[kernel] * (N - 2) ** 3
        kind = shape[0]
        assert kind in ("register", "staged", "bulk-copy", "flat")
        if kind == "register":
            tiles = dict(zip(("block", "kz", "narrow"), shape[1:]))
            got = B._kernel_shape(kernel, {"tiles": tiles, "stencil": {"sx": 0},
                                           "tma": {"rows": 0}, "xr": "column march"})
        elif kind == "bulk-copy":
            rows, planes, stages = shape[1:4]
            nodes = shape[4] if len(shape) > 4 else 1
            got = B._kernel_shape(kernel, {
                "tiles": {"block": 128, "kz": 1, "narrow": 0}, "stencil": {"sx": 0},
                "tma": {"rows": rows, "planes": planes, "stages": stages,
                        "kernels": 1 if kernel == "k_bicg_pv" else 2, "nodes": nodes},
                "xr": "column march"})
        elif kind == "flat":
            got = B._kernel_shape(kernel, {"tiles": {"block": 128, "kz": 1, "narrow": 0},
                                           "stencil": {"sx": 0}, "tma": {"rows": 0},
                                           "xr": "flat stream"})
        else:
            got = shape
        assert got == shape, (kernel, shape, got)
