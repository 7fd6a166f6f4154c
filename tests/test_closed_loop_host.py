"""The host side of the closed loop (the simulated vehicle, the obstacle
advance, the waypoint completion check) that the host-driven loop and the
benchmark's end-to-end path use (CPU only): the vehicle step equals the
oracle's Euler step of the kinematic bicycle (Sect. IV) and reduces to a
straight line without steering; points move at constant velocity; a
waypoint counts as reached only within every tolerance, the heading error
wrapped."""
import math

import numpy as np

from paper_1904_06680_gb300 import closed_loop, inputs


def test_plant_step_equals_the_oracle_euler_step(orc):
    rng = np.random.default_rng(4)
    for p in (inputs.planner(32), inputs.PAPER):
        for _ in range(200):
            z = np.array([rng.uniform(-50, 50), rng.uniform(-50, 50), rng.uniform(-7, 7), rng.uniform(-5, 15)])
            a = rng.uniform(-1, 1, 2)
            got = closed_loop.plant_step(p, np.concatenate([z, [0.3, -0.2]]), a)
            want = orc.euler_step(p, z, a)
            assert np.allclose(got[:4], want, rtol=1e-12, atol=1e-12), (got[:4], want)
            assert np.array_equal(got[4:], a)          # the applied controls become a_prev


def test_plant_step_straight_line():
    p = inputs.planner(16)
    s = np.array([1.0, 2.0, 0.5, 3.0, 0.0, 0.0])
    a = np.array([0.0, 0.5])                           # no steering, constant acceleration
    u = p["u_min"] + 0.75 * (p["u_max"] - p["u_min"])
    n = 30
    for _ in range(n):
        s = closed_loop.plant_step(p, s, a)
    dist = p["Ts"] * (n * 3.0 + u * p["Ts"] * n * (n - 1) / 2)
    assert math.isclose(s[0], 1.0 + dist * math.cos(0.5), rel_tol=1e-12)
    assert math.isclose(s[1], 2.0 + dist * math.sin(0.5), rel_tol=1e-12)
    assert s[2] == 0.5 and math.isclose(s[3], 3.0 + n * p["Ts"] * u, rel_tol=1e-12)


def test_advance_obstacles_constant_velocity():
    obs = np.array([[0.0, 0.0, 1.0, -2.0], [5.0, 5.0, 0.0, 0.0]])
    out = closed_loop.advance_obstacles(closed_loop.advance_obstacles(obs, 0.1), 0.1)
    assert np.allclose(out, [[0.2, -0.4, 1.0, -2.0], [5.0, 5.0, 0.0, 0.0]])
    assert np.array_equal(obs[0], [0.0, 0.0, 1.0, -2.0])       # the input is not modified


def test_reached_every_tolerance_in_the_vehicle_frame():
    eps = inputs.EPS                                   # (xi, eta, phi, v)
    s = np.array([10.0, 0.0, math.pi / 2, 1.0, 0.0, 0.0])      # facing +y
    # along the heading (+y) 0.9 m, across 0.2 m: inside
    assert closed_loop.reached(s, np.array([10.2, 0.9, math.pi / 2, 1.0]), eps)
    # across the heading beyond eta (0.25 m)
    assert not closed_loop.reached(s, np.array([10.3, 0.0, math.pi / 2, 1.0]), eps)
    # along the heading beyond xi (1 m)
    assert not closed_loop.reached(s, np.array([10.0, 1.1, math.pi / 2, 1.0]), eps)
    # heading error wrapped: pi/2 + 2 pi + 5 deg is within 10 deg
    assert closed_loop.reached(s, np.array([10.0, 0.0, math.pi / 2 + 2 * math.pi + math.radians(5), 1.0]), eps)
    assert not closed_loop.reached(s, np.array([10.0, 0.0, math.pi / 2 + math.radians(11), 1.0]), eps)
    # speed beyond 5 km/h
    assert not closed_loop.reached(s, np.array([10.0, 0.0, math.pi / 2, 1.0 + 1.5]), eps)


def test_mission_advances_through_its_waypoints():
    wp = np.array([[0.0, 0.0, 0.0, 0.0], [5.0, 0.0, 0.0, 0.0]])
    m = closed_loop.Mission(wp, inputs.EPS)
    assert not m.done and np.array_equal(m.goal, wp[0])
    m.update(np.array([3.0, 0.0, 0.0, 0.0, 0, 0]))            # not there yet
    assert m.k == 0
    m.update(np.array([0.5, 0.1, 0.0, 0.0, 0, 0]))
    assert m.k == 1 and np.array_equal(m.goal, wp[1])
    m.update(np.array([5.0, 0.0, 0.0, 0.0, 0, 0]))
    assert m.done and np.array_equal(m.goal, wp[1])            # the last goal stays
    m.update(np.array([50.0, 0.0, 0.0, 0.0, 0, 0]))
    assert m.k == 2
