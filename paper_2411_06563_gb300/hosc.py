"""Python binding of libhosc.so (the C ABI declared in include/hosc.h), argument marshalling only.

The functions keep the C names (hosc_create, hosc_step, ...). ``Cavity`` is a small convenience
wrapper that owns one context and exchanges fields as numpy arrays of shape (N, N, N) indexed
[z, y, x] (x fastest, the library's layout). Every step of the method runs in the CUDA library;
there is no Python or CPU fallback: if the library is missing this module raises.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhosc.so")

# status codes
HOSC_OK, HOSC_EINVAL, HOSC_ENOMEM, HOSC_ECUDA, HOSC_ENOCONV, HOSC_EDIVERGED, HOSC_ESTEPLIMIT, \
    HOSC_ESTATE = range(8)
HOSC_FP64, HOSC_MIXED = 0, 1
# fields
(HOSC_U, HOSC_V, HOSC_W, HOSC_THETA, HOSC_P, HOSC_ETA, HOSC_LCOEF, HOSC_EU, HOSC_EV, HOSC_EW,
 HOSC_RHS_U, HOSC_RHS_V, HOSC_RHS_W, HOSC_RHS_THETA, HOSC_DX_U, HOSC_DX_V, HOSC_DX_W,
 HOSC_DX_THETA, HOSC_PREV_L, HOSC_PREV_U, HOSC_PREV_V, HOSC_PREV_W, HOSC_PREV_EU, HOSC_PREV_EV,
 HOSC_PREV_EW, HOSC_DIV) = range(26)
HOSC_A_MOM, HOSC_A_ENE = 26, 33   # + 0..6: centre, x+, x-, y+, y-, z+, z-
# stages
(HOSC_STAGE_VISCOSITY, HOSC_STAGE_SOURCES, HOSC_STAGE_RHS, HOSC_STAGE_SOLVE,
 HOSC_STAGE_UPDATE) = range(5)
# kernel classes for profiling
(HOSC_K_VISC, HOSC_K_SOURCES, HOSC_K_RHS, HOSC_K_BICG_PV, HOSC_K_BICG_ST, HOSC_K_BICG_XR,
 HOSC_K_UPDATE) = range(7)


class hosc_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
                ("n", ctypes.c_double), ("dt", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("theta_ref", ctypes.c_double), ("theta_init", ctypes.c_double),
                ("I2_eps", ctypes.c_double), ("phi", ctypes.c_double),
                ("tol_steady", ctypes.c_double), ("tol_div", ctypes.c_double),
                ("tol_lin", ctypes.c_double), ("max_lin_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("a_limit", ctypes.c_double), ("a_boost", ctypes.c_double),
                ("use_history", ctypes.c_int), ("auto_defect", ctypes.c_int),
                ("precond", ctypes.c_int), ("inner_max", ctypes.c_int),
                ("Ly", ctypes.c_double), ("Lz", ctypes.c_double), ("solver", ctypes.c_int),
                ("lambda_mode", ctypes.c_int), ("div_steady", ctypes.c_double)]


class hosc_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("lin_iters", ctypes.c_long),
                ("last_iters", ctypes.c_int * 4), ("res_steady", ctypes.c_double),
                ("div_max", ctypes.c_double), ("lin_res", ctypes.c_double),
                ("status", ctypes.c_int), ("inner_passes", ctypes.c_long),
                ("sys_iters", ctypes.c_long * 4), ("solve_iters", ctypes.c_long)]

    def as_dict(self):
        return dict(steps=self.steps, lin_iters=self.lin_iters, last_iters=list(self.last_iters),
                    res=self.res_steady, div_max=self.div_max, lin_res=self.lin_res,
                    status=self.status, inner_passes=self.inner_passes,
                    sys_iters=list(self.sys_iters), solve_iters=self.solve_iters)


class hosc_diag(ctypes.Structure):
    _fields_ = [("Nu_hot_max", ctypes.c_double), ("Nu_hot_mean", ctypes.c_double),
                ("Nu_cold_mean", ctypes.c_double), ("E_total", ctypes.c_double),
                ("E_HT", ctypes.c_double), ("E_FF", ctypes.c_double), ("Be", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hosc_pool_info(ctypes.Structure):
    _fields_ = [("active", ctypes.c_int), ("completed", ctypes.c_int),
                ("tuned_sizes", ctypes.c_int), ("bytes_used", ctypes.c_size_t),
                ("budget", ctypes.c_size_t), ("rounds", ctypes.c_long),
                ("captures", ctypes.c_long), ("capture_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


HOSC_POOL_STREAMS, HOSC_POOL_GRAPH, HOSC_POOL_PERSISTENT = 0, 1, 2


class HoscError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = "%s: %s (%d)" % (where, hosc_strerror(status), status)
        detail = hosc_last_error_detail()
        if detail and status in (HOSC_ECUDA, HOSC_ENOMEM):
            msg += " [" + detail + "]"
        super().__init__(msg)


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    """The loaded libhosc.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhosc.so not found at %s: build it with "
                           "`python -m paper_2411_06563_gb300.build`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "hosc_default_params": (ctypes.c_int, [ctypes.POINTER(hosc_params), ctypes.c_int,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "hosc_steady_params": (ctypes.c_int, [ctypes.POINTER(hosc_params), ctypes.c_int,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "hosc_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(hosc_params)]),
        "hosc_fp64_peak": (ctypes.c_int, [ctypes.c_int, _DP]),
        "hosc_create": (ctypes.c_int, [ctypes.POINTER(hosc_params), ctypes.POINTER(_P)]),
        "hosc_create_in": (ctypes.c_int, [ctypes.POINTER(hosc_params), _P, ctypes.c_size_t,
                                          ctypes.POINTER(_P)]),
        "hosc_destroy": (None, [_P]),
        "hosc_reset": (ctypes.c_int, [_P]),
        "hosc_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(hosc_info)]),
        "hosc_solve_steady": (ctypes.c_int, [_P, ctypes.c_long, ctypes.POINTER(hosc_info)]),
        "hosc_run_stage": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(hosc_info)]),
        "hosc_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(hosc_diag), _DP, _DP]),
        "hosc_get_field": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
        "hosc_set_field": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
        "hosc_clear_history": (ctypes.c_int, [_P]),
        "hosc_get_field_device": (ctypes.c_int, [_P, ctypes.c_int, _P]),
        "hosc_set_field_device": (ctypes.c_int, [_P, ctypes.c_int, _P]),
        "hosc_get_params": (ctypes.c_int, [_P, ctypes.POINTER(hosc_params)]),
        "hosc_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
        "hosc_profile_read": (ctypes.c_int, [_P, ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_long),
                                             _DP]),
        "hosc_kernel_launches": (ctypes.c_long, [_P]),
        "hosc_time_kernel": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _DP, _DP]),
        "hosc_set_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "hosc_get_tiles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
        "hosc_set_stencil_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "hosc_set_tma_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int]),
        "hosc_get_tma_tiles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
        "hosc_set_xr_form": (ctypes.c_int, [_P, ctypes.c_int]),
        "hosc_get_xr_form": (ctypes.c_int, [_P]),
        "hosc_set_krylov_merged": (ctypes.c_int, [_P, ctypes.c_int]),
        "hosc_get_krylov_merged": (ctypes.c_int, [_P]),
        "hosc_get_stencil_tiles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int)]),
        "hosc_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), _DP]),
        "hosc_set_phase": (ctypes.c_int, [_P, ctypes.c_int]),
        "hosc_bicgstab_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P),
                                                 ctypes.POINTER(_P), ctypes.POINTER(_P),
                                                 ctypes.c_double, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int), _P]),
        "hosc_get_phase": (ctypes.c_int, [_P]),
        "hosc_pool_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(_P)]),
        "hosc_pool_destroy": (None, [_P]),
        "hosc_pool_admit": (ctypes.c_int, [_P, ctypes.POINTER(hosc_params), ctypes.c_long,
                                           ctypes.POINTER(ctypes.c_int)]),
        "hosc_pool_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "hosc_pool_result": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(hosc_info), ctypes.POINTER(hosc_diag),
                                            ctypes.POINTER(_P)]),
        "hosc_pool_retire": (ctypes.c_int, [_P, ctypes.c_int]),
        "hosc_pool_stats": (ctypes.c_int, [_P, ctypes.POINTER(hosc_pool_info)]),
        "hosc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "hosc_last_error_detail": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(_DP) if a is not None else None


# ------------------------------------------------------------------ thin C-name wrappers

def hosc_strerror(status):
    return lib().hosc_strerror(int(status)).decode()


def hosc_last_error_detail():
    return lib().hosc_last_error_detail().decode()


def hosc_default_params(N, Ra, Pr=1.0, n=1.0, **overrides):
    p = hosc_params()
    st = lib().hosc_default_params(ctypes.byref(p), int(N), float(Ra), float(Pr), float(n))
    if st:
        raise HoscError(st, "hosc_default_params")
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def hosc_steady_params(N, Ra, Pr=1.0, n=1.0, **overrides):
    p = hosc_params()
    st = lib().hosc_steady_params(ctypes.byref(p), int(N), float(Ra), float(Pr), float(n))
    if st:
        raise HoscError(st, "hosc_steady_params")
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def hosc_fp64_peak(reps=10):
    out = ctypes.c_double()
    st = lib().hosc_fp64_peak(int(reps), ctypes.byref(out))
    return st, out.value


def hosc_workspace_bytes(p):
    return int(lib().hosc_workspace_bytes(ctypes.byref(p)))


def hosc_create(p):
    h = _P()
    st = lib().hosc_create(ctypes.byref(p), ctypes.byref(h))
    return st, h


def hosc_create_in(p, dev_ptr, nbytes):
    h = _P()
    st = lib().hosc_create_in(ctypes.byref(p), _P(dev_ptr), ctypes.c_size_t(nbytes), ctypes.byref(h))
    return st, h


def hosc_destroy(h):
    lib().hosc_destroy(h)


def hosc_reset(h):
    return lib().hosc_reset(h)


def hosc_step(h, nsteps):
    info = hosc_info()
    st = lib().hosc_step(h, int(nsteps), ctypes.byref(info))
    return st, info


def hosc_solve_steady(h, max_steps):
    info = hosc_info()
    st = lib().hosc_solve_steady(h, int(max_steps), ctypes.byref(info))
    return st, info


def hosc_run_stage(h, stage):
    info = hosc_info()
    st = lib().hosc_run_stage(h, int(stage), ctypes.byref(info))
    return st, info


def hosc_diagnostics(h, N, with_fields=False):
    d = hosc_diag()
    nu = np.empty(N)
    fields = np.empty((3, N, N, N)) if with_fields else None
    st = lib().hosc_diagnostics(h, ctypes.byref(d), _dp(nu), _dp(fields))
    return st, d, nu, fields


def hosc_get_field(h, which, out):
    return lib().hosc_get_field(h, int(which), _dp(out))


def hosc_set_field(h, which, arr):
    return lib().hosc_set_field(h, int(which), _dp(arr))


def hosc_clear_history(h):
    return lib().hosc_clear_history(h)


def hosc_get_field_device(h, which, dev_ptr):
    return lib().hosc_get_field_device(h, int(which), _P(dev_ptr))


def hosc_set_field_device(h, which, dev_ptr):
    return lib().hosc_set_field_device(h, int(which), _P(dev_ptr))


def hosc_get_params(h):
    p = hosc_params()
    st = lib().hosc_get_params(h, ctypes.byref(p))
    return st, p


def hosc_profile_enable(h, on=1):
    return lib().hosc_profile_enable(h, int(on))


def hosc_profile_read(h, kernel_id):
    ms = ctypes.c_double()
    n = ctypes.c_long()
    b = ctypes.c_double()
    st = lib().hosc_profile_read(h, int(kernel_id), ctypes.byref(ms), ctypes.byref(n),
                                 ctypes.byref(b))
    return st, ms.value, n.value, b.value


def hosc_time_kernel(h, kernel_id, reps):
    ms = ctypes.c_double()
    b = ctypes.c_double()
    st = lib().hosc_time_kernel(h, int(kernel_id), int(reps), ctypes.byref(ms), ctypes.byref(b))
    return st, ms.value, b.value


def hosc_set_tiles(h, kblock, kz, narrow=0):
    return lib().hosc_set_tiles(h, int(kblock), int(kz), int(narrow))


def hosc_get_tiles(h):
    """(status, kblock, kz, narrow)"""
    b = ctypes.c_int()
    z = ctypes.c_int()
    n = ctypes.c_int()
    st = lib().hosc_get_tiles(h, ctypes.byref(b), ctypes.byref(z), ctypes.byref(n))
    return st, b.value, z.value, n.value


def hosc_set_stencil_tiles(h, sx, sy, skz):
    return lib().hosc_set_stencil_tiles(h, int(sx), int(sy), int(skz))


def hosc_set_tma_tiles(h, tty, tkz, stages=3, kernels=3):
    return lib().hosc_set_tma_tiles(h, int(tty), int(tkz), int(stages), int(kernels))


def hosc_get_tma_tiles(h):
    """(status, rows, planes, stages, kernels)."""
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = lib().hosc_get_tma_tiles(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                  ctypes.byref(d))
    return st, a.value, b.value, c.value, d.value


def hosc_set_xr_form(h, flat):
    return lib().hosc_set_xr_form(h, int(flat))


def hosc_get_xr_form(h):
    return int(lib().hosc_get_xr_form(h))


def hosc_set_krylov_merged(h, merged):
    return lib().hosc_set_krylov_merged(h, int(merged))


def hosc_get_krylov_merged(h):
    return int(lib().hosc_get_krylov_merged(h))


def hosc_get_stencil_tiles(h):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = lib().hosc_get_stencil_tiles(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return st, a.value, b.value, c.value


def hosc_autotune(h, reps=5):
    b = ctypes.c_int()
    z = ctypes.c_int()
    ms = ctypes.c_double()
    st = lib().hosc_autotune(h, int(reps), ctypes.byref(b), ctypes.byref(z), ctypes.byref(ms))
    return st, b.value, z.value, ms.value


def hosc_pool_create(budget_bytes, steps_per_round=8, mode=HOSC_POOL_GRAPH, autotune=1):
    h = _P()
    st = lib().hosc_pool_create(int(budget_bytes), int(steps_per_round), int(mode),
                                int(autotune), ctypes.byref(h))
    return st, h


def hosc_pool_destroy(pool):
    lib().hosc_pool_destroy(pool)


def hosc_pool_admit(pool, params, max_steps):
    slot = ctypes.c_int(-1)
    st = lib().hosc_pool_admit(pool, ctypes.byref(params), int(max_steps), ctypes.byref(slot))
    return st, slot.value


def hosc_pool_run(pool, rounds, cap=256):
    done = (ctypes.c_int * max(cap, 1))()
    nd = ctypes.c_int(0)
    st = lib().hosc_pool_run(pool, int(rounds), done, int(cap), ctypes.byref(nd))
    return st, [done[q] for q in range(min(nd.value, cap))]


def hosc_pool_result(pool, slot):
    status = ctypes.c_int()
    info = hosc_info()
    diag = hosc_diag()
    ctx = _P()
    st = lib().hosc_pool_result(pool, int(slot), ctypes.byref(status), ctypes.byref(info),
                                ctypes.byref(diag), ctypes.byref(ctx))
    return st, status.value, info, diag, ctx


def hosc_pool_retire(pool, slot):
    return lib().hosc_pool_retire(pool, int(slot))


def hosc_pool_stats(pool):
    out = hosc_pool_info()
    st = lib().hosc_pool_stats(pool, ctypes.byref(out))
    return st, out


def hosc_kernel_launches(h):
    return int(lib().hosc_kernel_launches(h))


HOSC_NOALLOC_MAX_N = 41


def hosc_bicgstab_noalloc(N, weights, rhs, x, tol, max_iter, stream=None):
    """Allocation-free solve (see include/hosc.h): weights, rhs, x are sequences of device
    addresses (ints) of N^3 double arrays (14, 4 and 4 of them). Returns (status, iters[4])."""
    W = (_P * 14)(*[_P(a) for a in weights])
    R = (_P * 4)(*[_P(a) for a in rhs])
    X = (_P * 4)(*[_P(a) for a in x])
    its = (ctypes.c_int * 4)()
    st = lib().hosc_bicgstab_noalloc(int(N), W, R, X, float(tol), int(max_iter), its,
                                     _P(stream) if stream else None)
    return st, list(its)


def hosc_set_phase(h, phase):
    return lib().hosc_set_phase(h, int(phase))


def hosc_get_phase(h):
    return int(lib().hosc_get_phase(h))


# ------------------------------------------------------------------ convenience wrapper

class Cavity:
    """One cavity context. Fields are numpy float64 arrays of shape (N, N, N) indexed [z, y, x].

    ``workspace="torch"`` carves the device memory out of one PyTorch CUDA allocation (the
    library then owns no device memory); the default lets the library cudaMalloc it.
    """

    def __init__(self, params, workspace=None):
        self.params = params
        self.N = params.N
        self._ws = None
        if workspace == "torch":
            import torch
            nbytes = hosc_workspace_bytes(params)
            if nbytes == 0:
                raise HoscError(HOSC_EINVAL, "hosc_workspace_bytes")
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ptr = self._ws.data_ptr()
            ptr += (-ptr) % 256
            st, h = hosc_create_in(params, ptr, nbytes)
        else:
            st, h = hosc_create(params)
        if st:
            raise HoscError(st, "hosc_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            hosc_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st, where, allow=()):
        if st and st not in allow:
            raise HoscError(st, where)
        return st

    def reset(self):
        self._check(hosc_reset(self.h), "hosc_reset")

    def step(self, nsteps=1, allow=(HOSC_ENOCONV, HOSC_EDIVERGED)):
        st, info = hosc_step(self.h, nsteps)
        self._check(st, "hosc_step", allow)
        d = info.as_dict()
        d["call_status"] = st
        return d

    def solve_steady(self, max_steps, allow=(HOSC_ESTEPLIMIT,)):
        st, info = hosc_solve_steady(self.h, max_steps)
        self._check(st, "hosc_solve_steady", allow)
        d = info.as_dict()
        d["call_status"] = st
        return d

    def run_stage(self, stage):
        st, info = hosc_run_stage(self.h, stage)
        self._check(st, "hosc_run_stage")
        return info.as_dict()

    def get(self, which):
        out = np.empty((self.N,) * 3)
        self._check(hosc_get_field(self.h, which, out), "hosc_get_field")
        return out

    def set(self, which, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        if a.shape != (self.N,) * 3:
            raise ValueError("field must have shape (N, N, N)")
        self._check(hosc_set_field(self.h, which, a), "hosc_set_field")

    def clear_history(self):
        self._check(hosc_clear_history(self.h), "hosc_clear_history")

    def diagnostics(self, with_fields=False):
        st, d, nu, fields = hosc_diagnostics(self.h, self.N, with_fields)
        self._check(st, "hosc_diagnostics")
        out = d.as_dict()
        out["Nu_avg_z"] = nu
        if with_fields:
            out["E_HT_field"], out["E_FF_field"], out["E_local_field"] = fields
        return out

    def kernel_launches(self):
        return hosc_kernel_launches(self.h)
