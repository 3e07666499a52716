"""GB300 (sm_103a) MPPI hot path: Python binding of ``include/mppi.h``.

The binding marshals arguments only.  Device memory and streams come from
PyTorch (``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``);
every step of the method runs in the library's CUDA kernels.  When the library
is missing the calls raise instead of falling back to the CPU.

    ctl = MPPI.from_problem(problem)          # problem dict (see workloads.py)
    out = ctl.step(x0, u_nom)                 # CUDA tensors in, CUDA tensors out
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _build
from ._lib import (MPPIError, CostDesc, DynamicsDesc, Options, check, load,  # noqa: F401
                   MPPI_PREC_FP32, MPPI_PREC_BF16_MLP)

__all__ = ["build", "MPPI", "MPPIError", "MPPIStep", "mppi_sample_noise",
           "mppi_update_noalloc", "fp32_fma_probe", "library_path"]

library_path = _build.LIB_PATH


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    return _build.build(force=force, verbose=verbose)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, n, name):
    import torch
    if t is None:
        return
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor with {n} elements")


class MPPI:
    """One MPPI controller context (``mppi_create`` ... ``mppi_destroy``)."""

    def __init__(self, *, dyn_kind, integrator, nx, nu, dyn_params, cost_kind, cost_params,
                 K, T, dt, lam, sigma, beta=1, seed=0, cost_map=None,
                 precision=MPPI_PREC_FP32, block_threads=0, rollout_variant=0, checked=0):
        L = load()
        self._dyn_params = _f32(dyn_params)
        self._cost_params = _f32(cost_params)
        self._sigma = _f32(sigma)
        self._map = None if cost_map is None else _f32(cost_map)
        dyn = DynamicsDesc(int(dyn_kind), int(integrator), int(nx), int(nu),
                           _fptr(self._dyn_params), self._dyn_params.size)
        if self._map is not None:
            cost = CostDesc(int(cost_kind), _fptr(self._cost_params), self._cost_params.size,
                            _fptr(self._map), self._map.shape[0], self._map.shape[1])
        else:
            cost = CostDesc(int(cost_kind), _fptr(self._cost_params), self._cost_params.size,
                            None, 0, 0)
        opt = Options()
        L.mppi_default_options(ctypes.byref(opt))
        opt.beta = int(beta)
        opt.seed = int(seed) & (2**64 - 1)
        opt.precision = int(precision)
        opt.block_threads = int(block_threads)
        opt.rollout_variant = int(rollout_variant)
        opt.checked = int(checked)
        h = ctypes.c_void_p()
        st = L.mppi_create(ctypes.byref(dyn), ctypes.byref(cost), int(K), int(T), float(dt),
                           float(lam), _fptr(self._sigma), ctypes.byref(opt), ctypes.byref(h))
        check(st, "mppi_create")
        self._h = h
        self._stream_val = None  # the stream handle last given to mppi_set_stream
        self.K, self.T, self.nx, self.nu = int(K), int(T), int(nx), int(nu)
        self.lam = float(lam)

    def _use_stream(self, L, stream):
        """mppi_set_stream, skipped when the context already uses that stream."""
        import torch
        s = (torch.cuda.current_stream() if stream is None else stream).cuda_stream
        if s != self._stream_val:
            check(L.mppi_set_stream(self._h, ctypes.c_void_p(s)), "mppi_set_stream", self._h)
            self._stream_val = s

    @classmethod
    def from_problem(cls, p: dict, **kw):
        """Build from a problem dictionary of ``workloads.py``."""
        args = dict(dyn_kind=p["dyn_kind"], integrator=p["integrator"], nx=p["nx"], nu=p["nu"],
                    dyn_params=p["dyn_params"], cost_kind=p["cost_kind"],
                    cost_params=p["cost_params"], K=p["K"], T=p["T"], dt=p["dt"], lam=p["lam"],
                    sigma=p["sigma"], beta=p["beta"], seed=p["seed"], cost_map=p.get("map"))
        args.update(kw)
        return cls(**args)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().mppi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- stepping ---------------------------------------------------------
    def step_into(self, x0, u_nom, u_new, weights=None, stats=None, costs=None, stream=None):
        """``mppi_step`` on caller-allocated CUDA tensors (no allocation)."""
        L = load()
        _check_tensor(x0, self.nx, "x0")
        _check_tensor(u_nom, self.T * self.nu, "u_nom")
        _check_tensor(u_new, self.T * self.nu, "u_new")
        _check_tensor(weights, self.K, "weights")
        _check_tensor(stats, 4, "stats")
        _check_tensor(costs, self.K, "costs")
        self._use_stream(L, stream)
        st = L.mppi_step(self._h, _dptr(x0), _dptr(u_nom), _dptr(u_new), _dptr(weights),
                         _dptr(stats), _dptr(costs))
        check(st, "mppi_step", self._h)

    def step(self, x0, u_nom, want_weights=False, want_costs=False, stream=None):
        """One iteration; returns dict(u_new[T, nu], stats[4], weights?, costs?)."""
        import torch
        dev = x0.device
        u_nom = u_nom.reshape(-1)
        out = dict(u_new=torch.empty(self.T * self.nu, device=dev, dtype=torch.float32),
                   stats=torch.empty(4, device=dev, dtype=torch.float32))
        if want_weights:
            out["weights"] = torch.empty(self.K, device=dev, dtype=torch.float32)
        if want_costs:
            out["costs"] = torch.empty(self.K, device=dev, dtype=torch.float32)
        self.step_into(x0, u_nom, out["u_new"], out.get("weights"), out["stats"],
                       out.get("costs"), stream=stream)
        out["u_new"] = out["u_new"].view(self.T, self.nu)
        return out

    def step_host(self, x0, u_nom, stream=None):
        """``mppi_step_host``: numpy/pinned host arrays in and out (synchronous)."""
        L = load()
        x0 = _f32(x0)
        u_nom = _f32(u_nom).reshape(-1)
        u_new = np.empty(self.T * self.nu, dtype=np.float32)
        stats = np.empty(4, dtype=np.float32)
        self._use_stream(L, stream)
        check(L.mppi_step_host(self._h, _fptr(x0), _fptr(u_nom), _fptr(u_new), _fptr(stats)),
              "mppi_step_host", self._h)
        return u_new.reshape(self.T, self.nu), stats

    def step_host_ptr(self, x0_ptr, u_nom_ptr, u_new_ptr, stats_ptr=None, stream=None):
        """``mppi_step_host`` on raw host addresses (e.g. pinned torch tensors)."""
        L = load()
        self._use_stream(L, stream)
        st = L.mppi_step_host_addr(self._h, x0_ptr, u_nom_ptr, u_new_ptr, stats_ptr or None)
        check(st, "mppi_step_host", self._h)

    def set_params(self, dyn_params=None, cost_params=None):
        L = load()
        d = None if dyn_params is None else _f32(dyn_params)
        c = None if cost_params is None else _f32(cost_params)
        check(L.mppi_set_params(self._h, None if d is None else _fptr(d),
                                None if c is None else _fptr(c)), "mppi_set_params", self._h)

    def set_params_device(self, dyn_params=None, cost_params=None, stream=None):
        """``mppi_set_params_device``: new parameter arrays from CUDA float32
        tensors, copied device to device on the stream (no host sync)."""
        L = load()
        _check_tensor(dyn_params, len(self._dyn_params), "dyn_params")
        _check_tensor(cost_params, len(self._cost_params), "cost_params")
        self._use_stream(L, stream)
        check(L.mppi_set_params_device(self._h, _dptr(dyn_params), _dptr(cost_params)),
              "mppi_set_params_device", self._h)

    def backward(self, grad_u_new, stream=None):
        """``mppi_step_backward``: gradient of sum(grad_u_new * u_new) of the last
        step w.r.t. (Q[4], R, l, m_cart); returns a CUDA tensor of 7."""
        import torch
        L = load()
        g = grad_u_new.reshape(-1).contiguous()
        _check_tensor(g, self.T * self.nu, "grad_u_new")
        out = torch.empty(7, device=g.device, dtype=torch.float32)
        self._use_stream(L, stream)
        check(L.mppi_step_backward(self._h, _dptr(g), _dptr(out)), "mppi_step_backward", self._h)
        return out

    @property
    def counter(self) -> int:
        v = ctypes.c_uint64()
        check(load().mppi_get_counter(self._h, ctypes.byref(v)), "mppi_get_counter", self._h)
        return int(v.value)

    @counter.setter
    def counter(self, value: int):
        check(load().mppi_set_counter(self._h, int(value) & (2**64 - 1)), "mppi_set_counter",
              self._h)

    def set_iterations(self, iterations: int, step_size: float = 1.0):
        """Algorithm 1's outer loop and the DMD-MPC step size (Sec. V-B): each
        step runs ``iterations`` rounds, moving the mean by
        u <- (1 - step_size) u + step_size * (weighted mean of the samples)."""
        check(load().mppi_set_iterations(self._h, int(iterations), float(step_size)),
              "mppi_set_iterations", self._h)

    def set_cem(self, top_k_fraction: float):
        """Cross-entropy-method weights (the lowest-cost fraction of the samples,
        equally weighted) instead of MPPI's; 0 returns to MPPI."""
        check(load().mppi_set_cem(self._h, float(top_k_fraction)), "mppi_set_cem", self._h)

    def nominal_trajectory(self, x0, u, stream=None):
        """States [T+1, nx] of x0 under the control sequence u, without noise."""
        import torch
        L = load()
        _check_tensor(x0, self.nx, "x0")
        _check_tensor(u, self.T * self.nu, "u")
        traj = torch.empty((self.T + 1, self.nx), dtype=torch.float32, device=x0.device)
        self._use_stream(L, stream)
        check(L.mppi_nominal_trajectory(self._h, _dptr(x0), _dptr(u), _dptr(traj)),
              "mppi_nominal_trajectory", self._h)
        return traj

    def shift(self, u, s: int, stream=None):
        """The control sequence advanced by s steps, the last s holding u[T-1]."""
        import torch
        L = load()
        _check_tensor(u, self.T * self.nu, "u")
        out = torch.empty_like(u)
        self._use_stream(L, stream)
        check(L.mppi_shift(self._h, _dptr(u), int(s), _dptr(out)), "mppi_shift", self._h)
        return out

    def profile(self, enable: bool):
        """Start (clearing the record) or stop per-kernel event timing."""
        check(load().mppi_profile(self._h, 1 if enable else 0), "mppi_profile", self._h)

    def profile_read(self):
        """{slot: (total_ms, launches)} for slots rollout, update, adjoint."""
        ms = (ctypes.c_float * 4)()
        n = (ctypes.c_int * 4)()
        check(load().mppi_profile_read(self._h, ms, n), "mppi_profile_read", self._h)
        names = ("rollout", "update", "adjoint", "other")
        return {names[i]: (float(ms[i]), int(n[i])) for i in range(4)}

    def poll_status(self) -> int:
        """Device status word since the last poll (0 = MPPI_OK); does not raise."""
        return int(load().mppi_poll_status(self._h))


def mppi_sample_noise(seed, step, K, Q, bits=None, z=None, stream=None):
    """Raw Philox words (uint32 stored in an int32 tensor) and normals the kernels use."""
    L = load()
    st = L.mppi_sample_noise(int(seed) & (2**64 - 1), int(step) & (2**64 - 1), int(K), int(Q),
                             _dptr(bits), _dptr(z), _stream_handle(stream))
    check(st, "mppi_sample_noise")


def fp32_fma_probe(pair=False, iters=200000):
    """Measured FP32 FMA rate of the current device (``mppi_fp32_fma_probe``):
    returns (TFLOP/s, milliseconds of the timed launch)."""
    L = load()
    ms = ctypes.c_float()
    fl = ctypes.c_double()
    check(L.mppi_fp32_fma_probe(1 if pair else 0, int(iters), ctypes.byref(ms), ctypes.byref(fl)),
          "mppi_fp32_fma_probe")
    return fl.value / (ms.value * 1e-3) / 1e12, ms.value


NOALLOC_MAX_K = 65536
NOALLOC_MAX_TNU = 4096


def mppi_update_noalloc(costs, lam, sigma, seed, step, u_nom, u_new, weights=None, stats=None,
                        stream=None):
    """Weights and control update from caller-computed costs without any device
    allocation (``mppi_update_noalloc``), for callers that cannot allocate GPU
    memory, e.g. a real-time control loop.  All tensors are caller-owned CUDA
    float32; K <= 65536 and T * nu <= 4096."""
    L = load()
    K = costs.numel()
    nu = len(sigma)
    TN = u_nom.numel()
    if K < 1 or K > NOALLOC_MAX_K or TN > NOALLOC_MAX_TNU or TN % nu:
        raise MPPIError(1, "mppi_update_noalloc",
                        f"K must be in [1, {NOALLOC_MAX_K}] and T*nu <= {NOALLOC_MAX_TNU}")
    _check_tensor(costs, K, "costs")
    _check_tensor(u_nom, TN, "u_nom")
    _check_tensor(u_new, TN, "u_new")
    _check_tensor(weights, K, "weights")
    _check_tensor(stats, 4, "stats")
    sig = _f32(sigma)
    st = L.mppi_update_noalloc(_dptr(costs), K, TN // nu, nu, float(lam), _fptr(sig),
                               int(seed) & (2**64 - 1), int(step) & (2**64 - 1), _dptr(u_nom),
                               _dptr(u_new), _dptr(weights), _dptr(stats),
                               _stream_handle(stream))
    check(st, "mppi_update_noalloc")


# ---------------------------------------------------------------------------
# differentiable step (cart-pole + quadratic cost + Euler)
# ---------------------------------------------------------------------------
def _theta_params(ctl_params, theta):
    """Full (dyn_params, cost_params) device arrays with theta = (Q[4], R, l, m_c)
    written into the cart-pole layouts [m_c, m_p, l, g] and [Q, R, goal, s]."""
    import torch
    dyn0, cost0 = ctl_params
    dyn = torch.stack([theta[6], dyn0[1], theta[5], dyn0[3]])
    cost = torch.cat([theta[0:5], cost0[5:]])
    return dyn.contiguous(), cost.contiguous()


class MPPIStep:
    """``torch.autograd.Function`` over one MPPI step of a cart-pole context:
    u_new = MPPIStep.apply(theta, x0, u_nom, ctl) with theta = (Q[4], R, l, m_c)
    as a CUDA float32 tensor.  The backward calls ``mppi_step_backward`` (the
    adjoint kernels) at the same noise; call it before the next step on ``ctl``.
    """

    _fn = None

    @classmethod
    def apply(cls, theta, x0, u_nom, ctl):
        if cls._fn is None:
            cls._fn = _make_step_function()
        return cls._fn.apply(theta, x0, u_nom, ctl)


def _make_step_function():
    import torch

    class _Step(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, x0, u_nom, ctl):
            th = theta.detach().to(torch.float32).contiguous()
            base = getattr(ctl, "_theta_base", None)
            if base is None or base[0].device != th.device:
                base = (torch.tensor(ctl._dyn_params, device=th.device),
                        torch.tensor(ctl._cost_params, device=th.device))
                ctl._theta_base = base
            dyn, cost = _theta_params(base, th)
            # device-to-device on the stream: theta never goes through the host
            ctl.set_params_device(dyn, cost)
            out = ctl.step(x0, u_nom)
            ctx.ctl = ctl
            ctx.counter = ctl.counter
            return out["u_new"]

        @staticmethod
        def backward(ctx, grad_u_new):
            if ctx.ctl.counter != ctx.counter:
                raise RuntimeError("MPPIStep.backward: the context stepped again after forward")
            g = ctx.ctl.backward(grad_u_new.contiguous().to(torch.float32))
            return g, None, None, None

    return _Step


# ---------------------------------------------------------------------------
# batched instances (mppi_batch_*)
# ---------------------------------------------------------------------------
class MPPIBatch:
    """Many independent MPPI instances stepped by one graph launch.

    ``problems`` are problem dictionaries (``workloads.py``); the batch owns
    one device buffer each for all x0, u_nom, u_new and statistics (slices
    per instance), created from the problems' x0 / u_nom.
    """

    def __init__(self, problems, block_threads=0, device="cuda"):
        import torch
        from ._lib import InstanceDesc
        L = load()
        self.n = len(problems)
        self.problems = problems
        self._keep = []
        nx = [int(p["nx"]) for p in problems]
        tn = [int(p["T"]) * int(p["nu"]) for p in problems]
        self.x0 = torch.tensor(np.concatenate([np.asarray(p["x0"], np.float32) for p in problems]),
                               device=device)
        self.u_nom = torch.tensor(np.concatenate(
            [np.asarray(p["u_nom"], np.float32).reshape(-1) for p in problems]), device=device)
        self.u_new = torch.zeros_like(self.u_nom)
        self.stats = torch.zeros(4 * self.n, device=device)
        self._xo = np.concatenate([[0], np.cumsum(nx)]).astype(int)
        self._uo = np.concatenate([[0], np.cumsum(tn)]).astype(int)
        descs = (InstanceDesc * self.n)()
        for i, p in enumerate(problems):
            dyn = _f32(p["dyn_params"])
            cost = _f32(p["cost_params"])
            sig = _f32(p["sigma"])
            self._keep += [dyn, cost, sig]
            d = descs[i]
            d.dyn = DynamicsDesc(int(p["dyn_kind"]), int(p["integrator"]), int(p["nx"]),
                                 int(p["nu"]), _fptr(dyn), dyn.size)
            d.cost = CostDesc(int(p["cost_kind"]), _fptr(cost), cost.size, None, 0, 0)
            d.K, d.T = int(p["K"]), int(p["T"])
            d.dt, d.lambda_ = float(p["dt"]), float(p["lam"])
            d.sigma = _fptr(sig)
            d.seed = int(p["seed"]) & (2**64 - 1)
            d.beta = int(p["beta"])
            d.x0_d = self.x0.data_ptr() + 4 * int(self._xo[i])
            d.u_nom_d = self.u_nom.data_ptr() + 4 * int(self._uo[i])
            d.u_new_d = self.u_new.data_ptr() + 4 * int(self._uo[i])
            d.stats_d = self.stats.data_ptr() + 16 * i
        opt = Options()
        L.mppi_default_options(ctypes.byref(opt))
        opt.block_threads = int(block_threads)
        h = ctypes.c_void_p()
        check(L.mppi_batch_create(self.n, descs, ctypes.byref(opt), ctypes.byref(h)),
              "mppi_batch_create")
        self._h = h

    def step(self, stream=None):
        check(load().mppi_batch_step(self._h, _stream_handle(stream)), "mppi_batch_step")

    def latency_ms(self, stream=None):
        out = (ctypes.c_float * self.n)()
        check(load().mppi_batch_latency(self._h, _stream_handle(stream), out), "mppi_batch_latency")
        return np.array(out[:], dtype=np.float64)

    def info(self):
        out = (ctypes.c_int * 4)()
        check(load().mppi_batch_info(self._h, out), "mppi_batch_info")
        return dict(block_threads=out[0], grid=out[1], rollout_items=out[2], update_items=out[3])

    def u_new_of(self, i):
        p = self.problems[i]
        return self.u_new[self._uo[i]:self._uo[i + 1]].view(int(p["T"]), int(p["nu"]))

    def stats_of(self, i):
        return self.stats[4 * i:4 * i + 4]

    def samples_of(self, i, stream=None):
        """Instance i's per-sample costs and weights of the last step
        (``mppi_batch_samples``), as two CUDA tensors of K_i."""
        import torch
        K = int(self.problems[i]["K"])
        costs = torch.empty(K, dtype=torch.float32, device=self.u_new.device)
        weights = torch.empty_like(costs)
        check(load().mppi_batch_samples(self._h, int(i), _dptr(costs), _dptr(weights),
                                        _stream_handle(stream)), "mppi_batch_samples")
        return costs, weights

    def close(self):
        if getattr(self, "_h", None):
            load().mppi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
