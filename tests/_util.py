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


# --------------------------------------------------------------------------
# Per-sample cost comparison with the FP64 oracle, aware of decision flips.
#
# FP32 cost accumulation: the kernels carry the state in FP32 (one rounding
# per operation, errors growing at most about linearly over the T steps of a
# stable rollout) and sum the running cost with Neumaier compensation (2 u).
# The per-sample bound is therefore |S_gpu - S_oracle| <= (T + 8) u max(1, |S|)
# with u = 2^-24 (measured on GB300: at most 0.16 T u on every FP32 model),
# plus, for costmap costs, the FP32 resolution of the map coordinate, and for
# the ring cost of Eq. 25 the cancellation in its momentum term
# (cost_abs_extra).
# BF16 MLP operands (unit roundoff 2^-9) perturb the residual r, whose share
# of the state derivative is about 0.4 dt per step: aligned over T = 100 steps
# that moves the speed by up to ~3e-3 and the cost by up to ~1e-3 relative,
# the stated BF16 bound (measured: 3e-5).
#
# Integer decisions (the sphere crash test, the ring indicators of Eq. 25) are
# taken by the oracle in FP64 on its own state.  The GPU decides on its FP32
# state, which differs from the oracle's by at most dp = (T + 8) u X (the same
# budget as the costs; X bounds |position|), so it can decide a step the other
# way only if the oracle's margin |min_i |p - c_i|^2 - r_i^2| (or
# |r^2 - r_in^2|, |r^2 - r_out^2|) is below
#   delta = 2 sqrt(d) R dp + d dp^2 + 8 u R^2
# (d = 2 or 3 coordinates, R the largest radius).  A sample whose cost differs
# by n != 0 whole jumps (c_crash or c_ring) must have margin <= delta, and its
# remaining difference must satisfy the cost bound.
# --------------------------------------------------------------------------
U32 = 2.0 ** -24
BF16_COST_REL = 1e-3


def cost_rel_bound(p, bf16=False):
    return BF16_COST_REL if bf16 else (p["T"] + 8) * U32


def cost_abs_extra(p):
    """Absolute bound added for costmap costs.  The FP32 lookup forms the
    cell coordinate g = (x - x_min) / cell - 1/2 of a map G cells wide, which
    it holds to about 2 G u cells per axis; the bilinear value then moves by
    at most that times the largest difference D between neighbouring texels,
    on each of the two axes.  Over the T running costs and the terminal cost:
    (T + 1) c_map 4 G u D."""
    import workloads as W
    if p["cost_kind"] == W.COST_CIRCLE:
        # Eq. 25's speed and angular-momentum terms c_v |v_des - |v|| and
        # c_h |h_des - (x v_y - y v_x)| cancel: their FP32 error is about
        # 4 u times the size of the products (|x|, |v| <= 4 on these
        # workloads), not of the small result.
        C = p["cost_params"]
        X = V = 4.0
        return p["T"] * 4 * U32 * (abs(C[4]) * V + abs(C[6]) * 2 * X * V)
    if p["cost_kind"] not in (W.COST_COSTMAP_SPEED, W.COST_GOAL_COSTMAP) or p.get("map") is None:
        return 0.0
    M = np.asarray(p["map"], np.float64)
    D = max(np.abs(np.diff(M, axis=0)).max(), np.abs(np.diff(M, axis=1)).max())
    G = max(M.shape)
    c_map = p["cost_params"][0] if p["cost_kind"] == W.COST_COSTMAP_SPEED else p["cost_params"][2]
    return (p["T"] + 1) * abs(c_map) * 4 * G * U32 * D


def decision_model(p):
    """(jump, delta) for costs with integer decisions, else None."""
    import workloads as W
    T = p["T"]
    dp = (T + 8) * U32
    if p["cost_kind"] == W.COST_QUAD_OBSTACLES:
        C = p["cost_params"]
        base = 2 * p["nx"] + p["nu"] + 1
        n = int(C[base])
        if n == 0:
            return None
        R = float(np.max(C[base + 2 + 3:base + 2 + 4 * n:4]))
        X, d = 32.0, 3
        jump = float(C[base + 1])
    elif p["cost_kind"] == W.COST_CIRCLE:
        C = p["cost_params"]
        R, X, d, jump = float(C[1]), 32.0, 2, float(C[2])
    else:
        return None
    dp *= X
    delta = 2.0 * np.sqrt(d) * R * dp + d * dp * dp + 8 * U32 * R * R
    return jump, delta


def is_magnitude(p, step=0, u_nom=None):
    """Per sample, lambda sum_t sum_j |(v - u/2) u| / sigma^2: the size of the
    importance-sampling terms, which can cancel against the running cost (S
    then is small while its FP32 error scales with these terms)."""
    import oracle
    u = np.asarray(p["u_nom"] if u_nom is None else u_nom, np.float64).reshape(p["T"], p["nu"])
    sig = np.asarray(p["sigma"], np.float64)
    if not p["beta"] or not np.any(u) or not np.any(sig > 0):
        return 0.0
    z = oracle.normals(p["seed"], step, p["K"], p["T"], p["nu"])
    v = u[None] + sig[None, None, :] * z
    iv = np.where(sig > 0, 1.0 / np.where(sig > 0, sig, 1.0) ** 2, 0.0)
    return p["lam"] * np.sum(np.abs((v - 0.5 * u[None]) * u[None]) * iv[None, None, :], axis=(1, 2))


def check_costs(p, g_S, o_S, margins=None, bf16=False, step=0, u_nom=None):
    """Every sample's cost against the oracle's (see the derivation above),
    relative to max(1, |S|, size of the importance-sampling terms).
    Returns (max relative residual, boolean mask of flipped samples)."""
    import oracle
    g_S = np.asarray(g_S, np.float64)
    o_S = np.asarray(o_S, np.float64)
    fin_g, fin_o = np.isfinite(g_S), np.isfinite(o_S)
    assert np.array_equal(fin_g, fin_o), "finite costs differ"
    dS = np.where(fin_o, g_S - o_S, 0.0)
    scale = np.maximum(1.0, np.maximum(np.abs(np.where(fin_o, o_S, 0)),
                                       np.abs(np.where(fin_g, g_S, 0))))
    scale = np.maximum(scale, is_magnitude(p, step, u_nom))
    flipped = np.zeros(len(o_S), bool)
    dm = decision_model(p)
    if dm is not None:
        jump, delta = dm
        n = np.rint(dS / jump)
        flipped = n != 0
        if flipped.any():
            if margins is None:
                margins = oracle.decision_margins(p, step=step, n_threads=n_threads())
            elif callable(margins):
                margins = margins()
            bad = flipped & ~(margins <= delta)
            assert not bad.any(), (
                f"cost decisions differ on samples {np.nonzero(bad)[0][:10]} whose margins "
                f"{margins[bad][:10]} exceed the FP32 bound {delta:.3g}")
        dS = dS - n * jump
    rel = np.abs(dS) / scale
    bound = cost_rel_bound(p, bf16) + cost_abs_extra(p) / scale
    worst = int(np.argmax(rel / bound))
    assert rel[worst] <= bound[worst], (
        f"sample {worst}: |dS|/max(1,|S|) = {rel[worst]:.3g} > {bound[worst]:.3g} "
        f"(S_gpu {g_S[worst]}, S_oracle {o_S[worst]})")
    return float(rel.max()), flipped


def cost_propagation(p, g_S, o_S, eps):
    """|u(S_gpu) - u(S_oracle)| per (t, j): how far the oracle's own FP64
    weighting and update move u_new when given the GPU's costs instead of its
    own, i.e. the part of the end-to-end difference that the per-sample cost
    differences (each checked by ``check_costs``, flipped decisions included)
    account for.  It is small when the weights are well conditioned; when a
    few samples share the weight and S / lambda is large, FP32 cost
    resolution alone moves u_new by more than 1e-4 sigma."""
    import oracle
    w_g, _, cg = oracle.weights(g_S, p["lam"])
    w_o, _, co = oracle.weights(o_S, p["lam"])
    if cg or co:
        return 0.0
    return np.abs(np.einsum("k,ktj->tj", w_g - w_o, eps))
