"""Seeded synthetic inputs shaped like the paper's cavity runs (no arithmetic of the method here).

The paper's workloads are its own simulations of the differentially heated cube (Sec. 2.1, 3, 4):
grids 11^3..91^3, Ra 1e2..1e5, n 0.75..1.25, Pr 0.71 / 1. There is no dataset; these generators
stand in for developed flow states and for the batched / served request mixes:

* ``cavity_state``: no-slip velocity built from a few low Fourier modes under the wall envelope
  sin(pi x) sin(pi y) sin(pi z), amplitude ~0.15 sqrt(Ra) (the scale of the paper's Table 1 values
  at Ra = 1e4); temperature 1 - x plus a smooth perturbation vanishing on the hot and cold walls;
  a smooth pressure of size ~0.05 Ra.
* ``batch_mix``: N uniform in {21, 31, 41, 61}, log10 Ra uniform in [2, 5], n uniform in
  [0.75, 1.25] (seed 20241106).
* ``request_stream``: Poisson arrivals, N in {21, 31, ..., 101}, log10 Ra uniform in [2, 5],
  n in {0.75, 1.0, 1.25} (seed 20241107).
* ``steady_mix``: small cavities that reach steady state at dt = 0.02 (N in {17, 21}, log10 Ra
  uniform in [2, 3], n uniform in [0.9, 1.1]; seed 20241108), for the equal-accuracy comparison.
* ``perturbed``: a nearby state (a previous time level for the history terms).

Arrays are float64 of shape (N, N, N) indexed [z, y, x].
"""

import numpy as np


def _grid(N):
    x = np.linspace(0.0, 1.0, N)
    return np.meshgrid(x, x, x, indexing="ij")   # Z, Y, X


def _smooth(rng, Z, Y, X, modes=4):
    f = np.zeros_like(X)
    for _ in range(modes):
        kx, ky, kz = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        a = rng.standard_normal()
        f += a * (np.cos(np.pi * kx * X + ph[0]) * np.cos(np.pi * ky * Y + ph[1])
                  * np.cos(np.pi * kz * Z + ph[2]))
    return f / np.sqrt(modes)


def cavity_state(N, Ra, seed, vel_scale=None, theta_walls=True):
    """A seeded developed-looking state: dict with u, v, w, th, p."""
    rng = np.random.default_rng(seed)
    Z, Y, X = _grid(N)
    env = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    s = 0.15 * np.sqrt(max(Ra, 1.0)) if vel_scale is None else vel_scale
    u = s * env * _smooth(rng, Z, Y, X)
    v = s * env * _smooth(rng, Z, Y, X)
    w = 0.3 * s * env * _smooth(rng, Z, Y, X)
    th = 1.0 - X + 0.25 * np.sin(np.pi * X) * _smooth(rng, Z, Y, X)
    if theta_walls:
        th[:, :, 0] = 1.0
        th[:, :, -1] = 0.0
    p = 0.05 * max(Ra, 1.0) * _smooth(rng, Z, Y, X)
    out = dict(u=u, v=v, w=w, th=th, p=p)
    for k in ("u", "v", "w"):
        a = out[k]
        a[0, :, :] = a[-1, :, :] = 0.0
        a[:, 0, :] = a[:, -1, :] = 0.0
        a[:, :, 0] = a[:, :, -1] = 0.0
    return out


def perturbed(state, seed, rel=0.02):
    """A nearby state (e.g. the previous time level): each field plus rel * its max * smooth noise
    that keeps the velocity walls at zero and the hot/cold wall temperatures."""
    rng = np.random.default_rng(seed)
    N = state["u"].shape[0]
    Z, Y, X = _grid(N)
    env = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    out = {}
    for k, a in state.items():
        scale = rel * max(1e-12, float(np.max(np.abs(a))))
        d = scale * _smooth(rng, Z, Y, X)
        if k in ("u", "v", "w", "th"):
            d = d * env
        out[k] = a + d
    return out


def batch_mix(count=64, seed=20241106, sizes=(21, 31, 41, 61)):
    """Uneven cavities for a batched launch: list of dicts (N, Ra, n, Pr)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(dict(N=int(rng.choice(sizes)), Ra=float(10.0 ** rng.uniform(2.0, 5.0)),
                        n=float(rng.uniform(0.75, 1.25)), Pr=1.0))
    return out


def steady_mix(count=8, seed=20241108, sizes=(17, 21)):
    """Small cavities that reach steady state in a few thousand steps at dt = 0.02 (for the
    equal-accuracy comparison): list of dicts (N, Ra, n, Pr), Ra log-uniform in [1e2, 1e3],
    n uniform in [0.9, 1.1]."""
    rng = np.random.default_rng(seed)
    return [dict(N=int(rng.choice(sizes)), Ra=float(10.0 ** rng.uniform(2.0, 3.0)),
                 n=float(rng.uniform(0.9, 1.1)), Pr=1.0) for _ in range(count)]


def request_stream(count=2000, rate=1.0, seed=20241107, sizes=tuple(range(21, 102, 10)),
                   indices=(0.75, 1.0, 1.25), ra_log10=(2.0, 5.0)):
    """Poisson request stream: list of dicts (t_arrival, N, Ra, n, Pr) sorted by arrival."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for q in range(count):
        out.append(dict(t=float(t[q]), N=int(rng.choice(sizes)),
                        Ra=float(10.0 ** rng.uniform(*ra_log10)), n=float(rng.choice(indices)),
                        Pr=1.0))
    return out
