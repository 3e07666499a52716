"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import os

import numpy as np


def as_f32_problem(p):
    """The same problem with every float rounded to FP32, so the CUDA path
    (which receives FP32) and the FP64 oracle start from identical values."""
    q = dict(p)
    for key in ("dyn_params", "cost_params", "sigma", "x0", "u_nom", "map", "obstacles",
                "u_target"):
        if q.get(key) is not None:
            q[key] = np.asarray(q[key], dtype=np.float32).astype(np.float64)
    q["dt"] = float(np.float32(p["dt"]))
    q["lam"] = float(np.float32(p["lam"]))
    return q


def with_(p, **kw):
    q = dict(p)
    q.update(kw)
    for key in ("sigma", "x0", "u_nom"):
        if key in kw:
            q[key] = np.asarray(kw[key], dtype=np.float64)
    if "u_nom" in kw:
        q["u_nom"] = q["u_nom"].reshape(q["T"], q["nu"])
    return q


def n_threads():
    return max(1, os.cpu_count() or 1)
