"""Pins for the oracle's collision check, cost and best-sample selection.

* Collision (Eq. eq_Apsietc_collAvoidIneqs): against an independent
  point-in-rectangle test by corner cross products on a dense point grid,
  with constant-velocity extrapolation (Sect. II-D, items (i)-(iv)).
* Rigid-motion invariance: moving the whole world scene changes no cost and
  no collision flag.
* Selection: brute-force argmin with lowest index on ties; a collided sample
  never beats a free one; permuting parameter vectors permutes the costs;
  all-collided scenes fall back to the longest survivor.
"""
import math

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs


def _corners(p, x, y, phi):
    c, s = math.cos(phi), math.sin(phi)
    cx, cy = x + p["c_off"] * c, y + p["c_off"] * s
    hl, hw = p["half_len"], p["half_wid"]
    local = [(hl, hw), (-hl, hw), (-hl, -hw), (hl, -hw)]       # counter-clockwise
    return [(cx + c * a - s * b, cy + s * a + c * b) for a, b in local]


def _inside_cross(corners, q):
    """strictly inside a convex CCW polygon: every edge cross product > 0;
    also returns the smallest distance to an edge line."""
    dmin = math.inf
    inside = True
    for i in range(4):
        ax, ay = corners[i]
        bx, by = corners[(i + 1) % 4]
        ex, ey = bx - ax, by - ay
        cr = ex * (q[1] - ay) - ey * (q[0] - ax)
        dmin = min(dmin, abs(cr) / math.hypot(ex, ey))
        if not cr > 0:
            inside = False
    return inside, dmin


@pytest.mark.parametrize("preset", ["paper", "planner"])
def test_collision_vs_cross_products(orc, preset):
    p = dict(inputs.PAPER) if preset == "paper" else inputs.planner(16)
    rng = np.random.default_rng(5)
    for _ in range(12):
        x, y = rng.uniform(-5, 5, 2)
        phi = rng.uniform(-4, 4)
        tau = rng.uniform(0, 3)
        gx, gy = np.meshgrid(np.linspace(x - 4, x + 4, 41), np.linspace(y - 4, y + 4, 41))
        pts = np.stack([gx.ravel(), gy.ravel()], 1) + rng.normal(0, 1e-3, (41 * 41, 2))
        vel = rng.uniform(-2, 2, pts.shape)
        obs = np.concatenate([pts - tau * vel, vel], 1)   # at time tau they sit on the grid
        corners = _corners(p, x, y, phi)
        n_in = 0
        for j in range(len(pts)):
            want, dist = _inside_cross(corners, pts[j])
            if dist < 1e-9:
                continue
            got, _, _ = orc.collide(p, x, y, phi, obs[j:j + 1], tau=tau)
            assert got == want, (j, pts[j])
            n_in += want
        assert n_in > 20
        # whole set: flag is the OR, counts split by margin
        flag, n_clear, n_near = orc.collide(p, x, y, phi, obs, tau=tau, margin=1e-4)
        assert flag and n_clear > 0


def test_collision_strict_faces(orc):
    """A point exactly on a face is not a collision (strict '<')."""
    p = inputs.planner(16)
    hl, hw = p["half_len"], p["half_wid"]
    for q, want in [((hl, 0.0), False), ((0.0, hw), False), ((hl - 1e-9, hw - 1e-9), True),
                    ((-hl, 0.0), False), ((0.0, 0.0), True)]:
        obs = np.array([[q[0], q[1], 0.0, 0.0]])
        assert orc.collide(p, 0.0, 0.0, 0.0, obs)[0] == want, q


def _rigid(state, goal, obs, ang, dx, dy):
    c, s = math.cos(ang), math.sin(ang)
    R = np.array([[c, -s], [s, c]])
    st = state.copy()
    st[:2] = R @ state[:2] + [dx, dy]
    st[2] = state[2] + ang
    gl = goal.copy()
    gl[:2] = R @ goal[:2] + [dx, dy]
    gl[2] = goal[2] + ang
    ob = obs.copy()
    ob[:, :2] = obs[:, :2] @ R.T + [dx, dy]
    ob[:, 2:] = obs[:, 2:] @ R.T
    return st, gl, ob


def test_rigid_motion_invariance(orc):
    sc = inputs.tiny_scene(1, N=512, T=25, M=60)
    p = sc["preset"]
    a = orc.plan(p, sc["state"], sc["goal"], sc["obs"], sc["N"], sc["T"], sc["seed"], sc["t_index"])
    st, gl, ob = _rigid(sc["state"], sc["goal"], sc["obs"], 1.234, -17.0, 42.5)
    b = orc.plan(p, st, gl, ob, sc["N"], sc["T"], sc["seed"], sc["t_index"])
    fa, fb = a["first_hit"], b["first_hit"]
    assert (fa >= 0).sum() > 20 and (fa < 0).sum() > 20          # both kinds present
    agree = fa == fb
    assert agree.mean() > 0.995
    free = (fa < 0) & (fb < 0)
    np.testing.assert_allclose(a["costs"][free], b["costs"][free], rtol=1e-9)
    assert a["best_idx"] == b["best_idx"]
    # the world trajectory moves with the scene
    c, s = math.cos(1.234), math.sin(1.234)
    moved = a["traj"][:, :2] @ np.array([[c, s], [-s, c]]) + [-17.0, 42.5]
    np.testing.assert_allclose(b["traj"][:, :2], moved, atol=1e-9)


def test_argmin_and_costs(orc):
    sc = inputs.tiny_scene(2, N=300, T=20, M=40)
    p = sc["preset"]
    r = orc.plan(p, sc["state"], sc["goal"], sc["obs"], sc["N"], sc["T"], sc["seed"], sc["t_index"])
    costs, fh = r["costs"], r["first_hit"]
    assert np.all(np.isinf(costs[fh >= 0])) and np.all(np.isfinite(costs[fh < 0]))
    assert r["status"] == 0
    assert r["best_idx"] == int(np.argmin(costs))           # first minimum
    assert fh[r["best_idx"]] < 0
    assert r["best_cost"] == costs[r["best_idx"]]
    # re-rolled winner reproduces its cost from its trajectory and controls
    goal_ev, obs_ev = orc.frame_to_ev(sc["state"], sc["goal"], sc["obs"])
    th = orc.theta(sc["seed"], sc["t_index"], r["best_idx"], orc.n_theta(p)).astype(np.float64)
    np.testing.assert_array_equal(th, r["best_theta"])
    one = orc.rollout_theta(p, th[None], [0, 0, 0, sc["state"][3]], sc["state"][4:6], goal_ev, obs_ev, sc["T"])
    assert one["cost"][0] == r["best_cost"]
    np.testing.assert_array_equal(one["ctrl"][0], r["controls"])
    zT = one["traj"][0][-1]
    E = np.sum(one["ctrl"][0] ** 2)
    J = (p["w_pos"] * math.hypot(zT[0] - goal_ev[0], zT[1] - goal_ev[1])
         + p["w_phi"] * abs(math.remainder(zT[2] - goal_ev[2], 2 * math.pi))
         + p["w_v"] * abs(zT[3] - goal_ev[3]) + p["w_effort"] * E / sc["T"])
    assert abs(J - r["best_cost"]) < 1e-12 * max(1.0, J)


def test_permutation_and_ties(orc):
    sc = inputs.tiny_scene(3, N=64, T=15, M=30)
    p = sc["preset"]
    nt = orc.n_theta(p)
    goal_ev, obs_ev = orc.frame_to_ev(sc["state"], sc["goal"], sc["obs"])
    th = np.stack([orc.theta(sc["seed"], 0, n, nt) for n in range(64)]).astype(np.float64)
    z0 = [0, 0, 0, sc["state"][3]]
    a = orc.rollout_theta(p, th, z0, sc["state"][4:6], goal_ev, obs_ev, sc["T"], record=False)
    perm = np.random.default_rng(6).permutation(64)
    b = orc.rollout_theta(p, th[perm], z0, sc["state"][4:6], goal_ev, obs_ev, sc["T"], record=False)
    np.testing.assert_array_equal(a["cost"][perm], b["cost"])
    np.testing.assert_array_equal(a["first_hit"][perm], b["first_hit"])
    # identical parameter vectors tie; the plan must return the lowest index
    dup = np.concatenate([th[:5], th[:5]])
    c = orc.rollout_theta(p, dup, z0, sc["state"][4:6], goal_ev, obs_ev, sc["T"], record=False)
    np.testing.assert_array_equal(c["cost"][:5], c["cost"][5:])


def test_warm_start_replaces_sample_zero(orc):
    sc = inputs.tiny_scene(4, N=50, T=12, M=20)
    p = sc["preset"]
    nt = orc.n_theta(p)
    warm = np.zeros(nt)
    warm[-2:] = [0.0, math.atanh(0.1)]
    r = orc.plan(p, sc["state"], sc["goal"], sc["obs"], 50, 12, sc["seed"], 0, warm=warm)
    goal_ev, obs_ev = orc.frame_to_ev(sc["state"], sc["goal"], sc["obs"])
    one = orc.rollout_theta(p, warm[None], [0, 0, 0, sc["state"][3]], sc["state"][4:6], goal_ev, obs_ev, 12)
    assert r["costs"][0] == one["cost"][0]


def test_infeasible_fallback(orc):
    """Every sample collides: status INFEASIBLE and the winner is the sample
    whose first collision comes last (lowest index on ties)."""
    p = inputs.planner(16)
    rng = np.random.default_rng(7)
    # a dense ring of points 3.5-6 m around the start, all moving inwards at
    # 2 m/s: it closes over the start within the horizon
    ang = rng.uniform(-math.pi, math.pi, 3000)
    rad = rng.uniform(3.5, 6.0, 3000)
    obs = np.zeros((3000, 4))
    obs[:, 0] = rad * np.cos(ang)
    obs[:, 1] = rad * np.sin(ang)
    obs[:, 2] = -2.0 * np.cos(ang)
    obs[:, 3] = -2.0 * np.sin(ang)
    state = np.array([0.0, 0.0, 0.3, 2.0, 0.0, 0.0])
    goal = np.array([20.0, 0.0, 0.0, 0.0])
    r = orc.plan(p, state, goal, obs, 200, 40, 99, 0)
    fh = r["first_hit"]
    assert np.all(fh >= 0) and r["status"] == 2
    assert r["best_idx"] == int(np.argmax(fh))
    # a point inside the car at h = 0 makes everything collide at once
    obs2 = np.array([[0.5, 0.1, 0.0, 0.0]])
    r2 = orc.plan(p, state, goal, obs2, 64, 10, 1, 0)
    assert r2["status"] == 2 and np.all(r2["first_hit"] == 0) and r2["best_idx"] == 0


def test_no_obstacles_and_edge_sizes(orc):
    sc = inputs.tiny_scene(5, N=33, T=1, M=0)
    r = orc.plan(sc["preset"], sc["state"], sc["goal"], sc["obs"], 33, 1, sc["seed"], 0)
    assert r["status"] == 0 and np.all(r["first_hit"] == -1)
    with pytest.raises(ValueError):
        orc.plan(sc["preset"], sc["state"], sc["goal"], sc["obs"], 0, 5, 1, 0)


def test_tshc_rounds_never_worse(orc):
    """The hill climb's restart rounds keep the best so far as sample 0, so
    the best cost is non-increasing over rounds; with one round it is the
    plain plan step."""
    sc = inputs.tiny_scene(17, N=64, T=15, M=40, width=16, box=15.0)
    st, gl, ob = (np.asarray(sc[k], np.float32).astype(np.float64) for k in ("state", "goal", "obs"))
    r = orc.plan_tshc(sc["preset"], st, gl, ob, 64, 15, sc["seed"], sc["t_index"], 4, 0.3)
    h = r["history"]
    assert all(h[i + 1] <= h[i] for i in range(len(h) - 1)), h
    assert h[-1] < h[0]
    one = orc.plan_tshc(sc["preset"], st, gl, ob, 64, 15, sc["seed"], sc["t_index"], 1, 0.3)
    plain = orc.plan(sc["preset"], st, gl, ob, 64, 15, sc["seed"], sc["t_index"])
    assert one["best_cost"] == plain["best_cost"] and one["best_idx"] == plain["best_idx"]


def test_cost_from_final_state_and_controls(orc):
    """orc.cost (the cost of a rollout from its final state and its applied
    controls) equals the rollout's own cost for every collision-free sample,
    and in hand-worked cases: at the goal only the effort term remains; a
    3-4-5 offset, a heading error across the +-pi wrap and a speed error add
    their weighted magnitudes."""
    p = inputs.planner(16)
    sc = inputs.tiny_scene(5, N=64, T=15, M=40, width=16)
    st = np.asarray(sc["state"], np.float64)
    goal_ev, obs_ev = orc.frame_to_ev(st, np.asarray(sc["goal"], np.float64), np.asarray(sc["obs"], np.float64))
    o = orc.rollout_samples(p, sc["seed"], 0, np.arange(64, dtype=np.int32), [0, 0, 0, st[3]], st[4:6],
                            goal_ev, obs_ev, 15)
    free = np.flatnonzero(o["first_hit"] < 0)
    assert len(free) > 0
    for k in free:
        assert orc.cost(p, o["traj"][k][-1], o["ctrl"][k], goal_ev) == o["cost"][k]
    ctrl = np.array([[0.5, -0.5], [1.0, 0.0], [0.0, 0.0], [-0.25, 0.75]])      # E = 0.5 + 1 + 0 + 0.625
    g = np.array([3.0, 4.0, 3.0, 2.0])
    assert math.isclose(orc.cost(p, g, ctrl, g), p["w_effort"] * 2.125 / 4, rel_tol=1e-15)
    z = np.array([0.0, 0.0, -3.0, 5.0])                  # heading error 6 rad wraps to 6 - 2 pi
    want = (p["w_pos"] * 5.0 + p["w_phi"] * (2 * math.pi - 6.0) + p["w_v"] * 3.0
            + p["w_effort"] * 2.125 / 4)
    assert math.isclose(orc.cost(p, z, ctrl, g), want, rel_tol=1e-14)
