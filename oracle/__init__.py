"""ctypes front end of the FP64 MPPI oracle (``oracle/mppi_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg import this module; the CUDA product path never
does.  Problems are the plain dictionaries built by ``workloads.py``.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppi_oracle.c")
_LIB = os.path.join(_HERE, "libmppi_oracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mppi_oracle.h"))):
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o",
            _LIB + ".tmp"]
    try:
        subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:] + ["-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OracleProblem(ctypes.Structure):
    _fields_ = [
        ("dyn_kind", ctypes.c_int), ("integrator", ctypes.c_int),
        ("nx", ctypes.c_int), ("nu", ctypes.c_int),
        ("dyn_params", _dp), ("n_dyn_params", ctypes.c_int),
        ("cost_kind", ctypes.c_int),
        ("cost_params", _dp), ("n_cost_params", ctypes.c_int),
        ("map", _dp), ("map_h", ctypes.c_int), ("map_w", ctypes.c_int),
        ("K", ctypes.c_int), ("T", ctypes.c_int),
        ("dt", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("sigma", _dp), ("beta", ctypes.c_int),
        ("seed", ctypes.c_uint64), ("step", ctypes.c_uint64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.oracle_noise_block.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_uint32, _u32p, _dp]
        L.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, _dp]
        P = ctypes.POINTER(OracleProblem)
        L.oracle_deriv.argtypes = [P, _dp, _dp, _dp]
        L.oracle_dynamics_step.argtypes = [P, _dp, _dp, _dp]
        L.oracle_running_cost.argtypes = [P, _dp, _dp]
        L.oracle_running_cost.restype = ctypes.c_double
        L.oracle_terminal_cost.argtypes = [P, _dp]
        L.oracle_terminal_cost.restype = ctypes.c_double
        L.oracle_costmap_sample.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.oracle_costmap_sample.restype = ctypes.c_double
        L.oracle_rollout.argtypes = [P, _dp, _dp, _dp, _dp]
        L.oracle_rollout.restype = ctypes.c_double
        L.oracle_weights.argtypes = [ctypes.c_int, _dp, ctypes.c_double, _dp, _dp]
        L.oracle_mppi_step.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.oracle_mppi_grad_cartpole.argtypes = [P, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.oracle_mppi_iterate.argtypes = [P, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                          _dp, _dp, ctypes.c_int]
        L.oracle_nominal_trajectory.argtypes = [P, _dp, _dp, _dp]
        L.oracle_nominal_trajectory.restype = None
        L.oracle_shift.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]
        L.oracle_shift.restype = None
        L.oracle_cem_weights.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp]
        L.oracle_cem_step.argtypes = [P, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int]
        L.oracle_max_threads.argtypes = []
        L.oracle_decision_margins.argtypes = [P, _dp, _dp, _dp, ctypes.c_int]
    return _lib


def _ptr(a):
    if a is None:
        return ctypes.cast(None, _dp)
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Problem:
    """Keeps the numpy arrays alive while the C struct points into them."""

    def __init__(self, p: dict, step: int = 0):
        self.p = p
        self._keep = {k: np.ascontiguousarray(p[k], dtype=np.float64)
                      for k in ("dyn_params", "cost_params", "sigma")}
        m = p.get("map")
        self._keep["map"] = None if m is None else np.ascontiguousarray(m, dtype=np.float64)
        s = OracleProblem()
        s.dyn_kind, s.integrator = int(p["dyn_kind"]), int(p["integrator"])
        s.nx, s.nu = int(p["nx"]), int(p["nu"])
        s.dyn_params, s.n_dyn_params = _ptr(self._keep["dyn_params"]), len(self._keep["dyn_params"])
        s.cost_kind = int(p["cost_kind"])
        s.cost_params, s.n_cost_params = _ptr(self._keep["cost_params"]), len(self._keep["cost_params"])
        if self._keep["map"] is not None:
            s.map = _ptr(self._keep["map"])
            s.map_h, s.map_w = self._keep["map"].shape
        else:
            s.map = ctypes.cast(None, _dp)
        s.K, s.T = int(p["K"]), int(p["T"])
        s.dt, s.lambda_ = float(p["dt"]), float(p["lam"])
        s.sigma, s.beta = _ptr(self._keep["sigma"]), int(p["beta"])
        s.seed, s.step = int(p["seed"]) & (2**64 - 1), int(step) & (2**64 - 1)
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p),
                               out.ctypes.data_as(_u32p))
    return out


def noise_block(seed, step, k, q):
    bits = np.zeros(4, dtype=np.uint32)
    z = np.zeros(4)
    lib().oracle_noise_block(seed & (2**64 - 1), step & (2**64 - 1), k, q,
                             bits.ctypes.data_as(_u32p), _ptr(z))
    return bits, z


def normals(seed, step, K, T, nu):
    z = np.zeros((K, T, nu))
    lib().oracle_normals(seed & (2**64 - 1), step & (2**64 - 1), K, T, nu, _ptr(z))
    return z


def deriv(p, x, v):
    P = Problem(p)
    x = np.ascontiguousarray(x, float)
    v = np.ascontiguousarray(v, float)
    out = np.zeros(p["nx"])
    lib().oracle_deriv(P.ref, _ptr(x), _ptr(v), _ptr(out))
    return out


def dynamics_step(p, x, v):
    P = Problem(p)
    x = np.ascontiguousarray(x, float)
    v = np.ascontiguousarray(v, float)
    out = np.zeros(p["nx"])
    lib().oracle_dynamics_step(P.ref, _ptr(x), _ptr(v), _ptr(out))
    return out


def running_cost(p, y, v):
    P = Problem(p)
    return lib().oracle_running_cost(P.ref, _ptr(np.ascontiguousarray(y, float)),
                                     _ptr(np.ascontiguousarray(v, float)))


def terminal_cost(p, y):
    P = Problem(p)
    return lib().oracle_terminal_cost(P.ref, _ptr(np.ascontiguousarray(y, float)))


def costmap_sample(p, x, y):
    P = Problem(p)
    return lib().oracle_costmap_sample(P.ref, float(x), float(y))


def rollout(p, v, x0=None, u_nom=None):
    """Trajectory (T+1, nx) and total cost of one sample with controls v (T, nu)."""
    P = Problem(p)
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(p["u_nom"] if u_nom is None else u_nom, float)
    v = np.ascontiguousarray(v, float)
    traj = np.zeros((p["T"] + 1, p["nx"]))
    S = lib().oracle_rollout(P.ref, _ptr(x0), _ptr(u), _ptr(v), _ptr(traj))
    return traj, S


def weights(S, lam):
    S = np.ascontiguousarray(S, float)
    w = np.zeros(len(S))
    stats = np.zeros(4)
    st = lib().oracle_weights(len(S), _ptr(S), float(lam), _ptr(w), _ptr(stats))
    return w, stats, st


def mppi_step(p, step=0, n_threads=1, x0=None, u_nom=None, want_eps=False):
    """One MPPI iteration; returns dict(u_new, w, S, stats, status[, eps])."""
    P = Problem(p, step)
    K, T, nu = p["K"], p["T"], p["nu"]
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(p["u_nom"] if u_nom is None else u_nom, float)
    u_new = np.zeros((T, nu))
    w = np.zeros(K)
    S = np.zeros(K)
    stats = np.zeros(4)
    eps = np.zeros((K, T, nu)) if want_eps else None
    st = lib().oracle_mppi_step(P.ref, _ptr(x0), _ptr(u), _ptr(u_new), _ptr(w), _ptr(S),
                                _ptr(stats), _ptr(eps), int(n_threads))
    out = dict(u_new=u_new, w=w, S=S, stats=stats, status=st)
    if want_eps:
        out["eps"] = eps
    return out


def mppi_iterate(p, iterations, gamma, step=0, n_threads=1, x0=None, u_nom=None):
    """Algorithm 1 with I iterations and the DMD-MPC step size gamma (Sec. V-B);
    returns dict(u_new, w, S, stats, status) of the last iteration."""
    P = Problem(p, step)
    K, T, nu = p["K"], p["T"], p["nu"]
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(p["u_nom"] if u_nom is None else u_nom, float)
    u_new = np.zeros((T, nu))
    w = np.zeros(K)
    S = np.zeros(K)
    stats = np.zeros(4)
    st = lib().oracle_mppi_iterate(P.ref, _ptr(x0), _ptr(u), int(iterations), float(gamma),
                                   _ptr(u_new), _ptr(w), _ptr(S), _ptr(stats), int(n_threads))
    return dict(u_new=u_new, w=w, S=S, stats=stats, status=st)


def nominal_trajectory(p, u, x0=None):
    """States (T+1, nx) of x0 under the control sequence u (T, nu), no noise."""
    P = Problem(p)
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(u, float)
    traj = np.zeros((p["T"] + 1, p["nx"]))
    lib().oracle_nominal_trajectory(P.ref, _ptr(x0), _ptr(u), _ptr(traj))
    return traj


def shift(u, s):
    """u shifted by s steps, the last s steps holding the final control."""
    u = np.ascontiguousarray(u, float)
    T, nu = u.shape
    out = np.zeros_like(u)
    lib().oracle_shift(T, nu, _ptr(u), int(s), _ptr(out))
    return out


def cem_weights(S, n_elite):
    """Elite-set weights (1/|E| on the n_elite lowest costs, ties included)
    and |E| (-1 for bad arguments)."""
    S = np.ascontiguousarray(S, float)
    w = np.zeros(len(S))
    n = lib().oracle_cem_weights(len(S), _ptr(S), int(n_elite), _ptr(w))
    return w, n


def cem_step(p, top_k_fraction, step=0, n_threads=1, x0=None, u_nom=None):
    """One CEM iteration; returns dict(u_new, w, S, status)."""
    P = Problem(p, step)
    K, T, nu = p["K"], p["T"], p["nu"]
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(p["u_nom"] if u_nom is None else u_nom, float)
    u_new = np.zeros((T, nu))
    w = np.zeros(K)
    S = np.zeros(K)
    st = lib().oracle_cem_step(P.ref, _ptr(x0), _ptr(u), float(top_k_fraction), _ptr(u_new),
                               _ptr(w), _ptr(S), int(n_threads))
    return dict(u_new=u_new, w=w, S=S, status=st)


def mppi_grad_cartpole(p, G, step=0, n_threads=1, x0=None, u_nom=None):
    """d(sum G * u_new)/d(Q[4], R, l, m_c) at fixed noise."""
    P = Problem(p, step)
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(p["u_nom"] if u_nom is None else u_nom, float)
    G = np.ascontiguousarray(G, float)
    grad = np.zeros(7)
    st = lib().oracle_mppi_grad_cartpole(P.ref, _ptr(x0), _ptr(u), _ptr(G), _ptr(grad),
                                         int(n_threads))
    return grad, st


def decision_margins(p, step=0, n_threads=1, x0=None, u_nom=None):
    """Per-sample distance (min over t) of the cost's integer decisions (crash
    test, ring indicators) from their thresholds; +inf without such decisions."""
    P = Problem(p, step)
    x0 = np.ascontiguousarray(p["x0"] if x0 is None else x0, float)
    u = np.ascontiguousarray(p["u_nom"] if u_nom is None else u_nom, float)
    margin = np.zeros(p["K"])
    st = lib().oracle_decision_margins(P.ref, _ptr(x0), _ptr(u), _ptr(margin), int(n_threads))
    assert st == 0
    return margin
