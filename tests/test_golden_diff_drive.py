"""The diff-drive benchmark workload and the oracle against the paper's
table of algorithm parameters (Sec. V), stored under tests/golden/ with its
citation (no GPU).

The workload generator must use exactly the printed values, and the
oracle's dynamics must act on them: a command beyond the limits moves the
robot by the table's maximum speed and turn rate times dt in one Euler step.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "diff_drive_algorithm_parameters.txt")


def _table():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, value, _unit = line.split()
                out[name] = float(value)
    return out


def test_table_is_complete():
    t = _table()
    assert len(t) == 16
    assert t["min_velocity"] < 0 < t["max_velocity"]
    assert t["min_rotation"] == -t["max_rotation"]


def test_workload_uses_the_table():
    t = _table()
    p = W.diff_drive()
    assert p["dt"] == t["dt"]
    assert p["lam"] == t["lambda"]
    assert p["T"] == int(t["mpc_horizon"])
    np.testing.assert_array_equal(p["sigma"], [t["control_std_dev"]] * 2)
    # dynamics parameters [v_min, v_max, w_min, w_max]
    np.testing.assert_array_equal(
        p["dyn_params"], [t["min_velocity"], t["max_velocity"], t["min_rotation"], t["max_rotation"]])
    C = p["cost_params"]   # [c_goal, c_angle, c_obs, gx, gy, g_theta, x_min, y_min, cell]
    assert (C[0], C[1], C[2]) == (t["goal_distance_coeff"], t["goal_angle_coeff"], t["obstacle_cost"])
    assert C[8] == pytest.approx(t["map_resolution"], rel=1e-15)
    rows, cols = p["map"].shape
    assert cols * C[8] == pytest.approx(t["map_width"], rel=1e-12)
    assert rows * C[8] == pytest.approx(t["map_height"], rel=1e-12)
    # the map is centred on the origin: x in [x_min, x_min + width)
    assert C[6] == pytest.approx(-t["map_width"] / 2) and C[7] == pytest.approx(-t["map_height"] / 2)
    # wheel radius and length of 1 m: body velocities are the commands
    assert t["wheel_radius"] == 1.0 and t["wheel_length"] == 1.0


@pytest.mark.parametrize("heading", [0.0, math.pi / 3])
def test_oracle_moves_at_the_table_limits(oracle_lib, heading):
    t = _table()
    p = W.diff_drive(K=4, T=4)
    dt = t["dt"]
    for cmd, v, w in (([10.0, 10.0], t["max_velocity"], t["max_rotation"]),
                      ([-10.0, -10.0], t["min_velocity"], t["min_rotation"])):
        x1 = oracle.dynamics_step(p, [0.25, -0.5, heading], cmd)
        want = [0.25 + dt * v * math.cos(heading), -0.5 + dt * v * math.sin(heading), heading + dt * w]
        np.testing.assert_allclose(x1, want, rtol=0, atol=1e-15)
