"""The allocation-free solve entry point (hosc_bicgstab_noalloc) against the context's own
BiCGSTAB stage, through the C ABI.

Callers that cannot call cudaMalloc (hosts whose allocator or memory pool already owns the device
memory, solvers held to a device-memory budget fixed at start-up) pass their own input and output
arrays; the scratch of the solve lives in a fixed device array inside the library. Here the
inputs are the right-hand sides and operator weights a context computed for one step, copied into
caller-owned torch buffers, and the outputs must match the increments the context's solve
produced (relative 1e-12, the FP64 parity tolerance of the solve is 1e-9), on two calls in a row
with different grid sizes (the second call finds the first call's scratch).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2411_06563_gb300.hosc")
torch = pytest.importorskip("torch")
from paper_2411_06563_gb300 import inputs  # noqa: E402


def _context_solve(N, seed):
    p = H.hosc_default_params(N, 1e4, 1.0, 0.8)
    p.dt = 0.003
    p.lambda_ = 0.25 / (N - 1) ** 2 / p.dt
    p.tol_lin = 1e-11
    p.max_lin_iter = 2000
    st = inputs.cavity_state(N, 1e4, seed=seed)
    with H.Cavity(p) as cav:
        for name, which in (("u", H.HOSC_U), ("v", H.HOSC_V), ("w", H.HOSC_W),
                            ("th", H.HOSC_THETA), ("p", H.HOSC_P)):
            cav.set(which, st[name])
        for stage in (H.HOSC_STAGE_VISCOSITY, H.HOSC_STAGE_SOURCES, H.HOSC_STAGE_RHS):
            cav.run_stage(stage)
        weights = [cav.get(H.HOSC_A_MOM + q) for q in range(7)] + \
                  [cav.get(H.HOSC_A_ENE + q) for q in range(7)]
        rhs = [cav.get(H.HOSC_RHS_U + s) for s in range(4)]
        info = cav.run_stage(H.HOSC_STAGE_SOLVE)
        dx = [cav.get(H.HOSC_DX_U + s) for s in range(4)]
    return p, weights, rhs, dx, info


def _noalloc(N, p, weights, rhs):
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in weights + rhs]
    out = [torch.full((N, N, N), 7.0, dtype=torch.float64, device="cuda") for _ in range(4)]
    torch.cuda.synchronize()
    st, iters = H.hosc_bicgstab_noalloc(N, [t.data_ptr() for t in dev[:14]],
                                        [t.data_ptr() for t in dev[14:]],
                                        [t.data_ptr() for t in out], p.tol_lin, p.max_lin_iter)
    torch.cuda.synchronize()
    return st, iters, [t.cpu().numpy() for t in out]


def test_noalloc_solve_matches_context_solve_twice():
    torch.cuda.init()
    for N, seed in ((21, 3), (17, 4)):
        p, weights, rhs, dx_ctx, info = _context_solve(N, seed)
        st, iters, dx = _noalloc(N, p, weights, rhs)
        assert st == H.HOSC_OK
        assert iters == info["last_iters"]
        inner = (slice(1, -1),) * 3
        for a, b in zip(dx, dx_ctx):
            scale = np.max(np.abs(b[inner]))
            assert np.max(np.abs(a[inner] - b[inner])) <= 1e-12 * scale
            assert np.all(a[0] == 7.0) and np.all(a[:, :, -1] == 7.0)   # walls untouched


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = H.HOSC_NOALLOC_MAX_N + 1
    dummy = [1] * 14
    st, _ = H.hosc_bicgstab_noalloc(big, dummy, [1] * 4, [1] * 4, 1e-8, 10)
    assert st == H.HOSC_EINVAL
    st, _ = H.hosc_bicgstab_noalloc(4, dummy, [1] * 4, [1] * 4, 1e-8, 10)
    assert st == H.HOSC_EINVAL
