"""Pins of the oracle's two rollout variants (Sect. V): velocity constraints
imposed by discarding samples, and the goal offsets of the features taken in
the vehicle's frame at t+h instead of the EV frame at t.

* Speed limits against the closed form v_h = v0 + h Ts u of a constant
  acceleration (zero network weights, output biases atanh(a)).
* The discard step of random samples against the first out-of-range speed
  read off the same samples' unconstrained trajectories (the trajectory up
  to the discard is the same, so the two must agree).
* Body-frame features against a plain rotation of the offset, the special
  headings 0 and pi/2, and the unchanged first control (phi_t = 0 in the EV
  frame at t).
"""
import math

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs


def _zero_net_theta(p, a0, a1):
    nt = sum(o * i + o for i, o in zip(p["widths"][:-1], p["widths"][1:]))
    th = np.zeros(nt)
    th[-2] = math.atanh(a0)
    th[-1] = math.atanh(a1)
    return th


def _limits(p, lo, hi):
    q = dict(p)
    q.update(v_limits=1, v_min=lo, v_max=hi)
    return q


@pytest.mark.parametrize("v0,a1,lo,hi,want", [
    (5.0, 0.5, -1.0, 6.02, 7),      # v_h = 5 + 0.15 h > 6.02 first at h = 7
    (5.0, -0.5, 2.95, 9.0, 14),     # v_h = 5 - 0.15 h < 2.95 first at h = 14
    (-2.0, 1.0 - 1e-9, -3.0, 1.0, 11),  # reversing, then too fast forward
    (5.0, 0.5, 4.0, 9.0, -1),       # 5 + 0.15 * 20 = 8 stays inside
])
def test_speed_limit_closed_form(orc, v0, a1, lo, hi, want):
    """Constant acceleration u = 3 a1 from speed v0: the first h >= 1 with
    v0 + h Ts u outside [lo, hi] is the sample's first_hit; cost +inf."""
    p = _limits(inputs.planner(16), lo, hi)
    T = 20
    u = p["u_min"] + 0.5 * (a1 + 1) * (p["u_max"] - p["u_min"])
    h = np.arange(1, T + 1)
    v = v0 + h * p["Ts"] * u
    bad = np.nonzero((v < lo) | (v > hi))[0]
    assert (int(h[bad[0]]) if bad.size else -1) == want       # the case is what it claims
    r = orc.rollout_theta(p, _zero_net_theta(p, 0.0, a1)[None], [0, 0, 0, v0], [0.0, a1], [50, 3, 1, 0],
                          np.zeros((0, 4)), T)
    assert r["first_hit"][0] == want
    if want >= 0:
        assert math.isinf(r["cost"][0])
        # rows after the discard repeat its state; controls there are zero
        np.testing.assert_array_equal(r["traj"][0][want:], np.tile(r["traj"][0][want], (T + 1 - want, 1)))
        assert np.all(r["ctrl"][0][want:] == 0)
        np.testing.assert_allclose(r["traj"][0][want, 3], v0 + want * p["Ts"] * u, atol=1e-12)
    else:
        assert math.isfinite(r["cost"][0])


def test_initial_speed_is_not_discarded(orc):
    """The given speed at h = 0 is outside the limits, the first controlled
    state is inside: the sample is kept."""
    p = _limits(inputs.planner(16), 0.0, 12.0)
    r = orc.rollout_theta(p, _zero_net_theta(p, 0.0, -1.0 + 1e-12)[None], [0, 0, 0, 12.1], [0.0, -1.0],
                          [50, 3, 1, 0], np.zeros((0, 4)), 10)
    assert r["first_hit"][0] == -1
    assert orc.speed_violated(p, 12.1, 0) is False
    assert orc.speed_violated(p, 12.1, 1) is True
    assert orc.speed_violated(p, 12.0, 1) is False and orc.speed_violated(p, 0.0, 3) is False
    assert orc.speed_violated(p, float("nan"), 2) is True
    assert orc.speed_violated(dict(p, v_limits=0), 99.0, 2) is False


@pytest.mark.parametrize("width", [16, 32])
def test_discard_step_from_unconstrained_trajectories(orc, width):
    """Random samples in an obstacle scene: with limits, first_hit = the
    earlier of the unconstrained first collision and the first h >= 1 whose
    unconstrained speed is out of range; the free samples' costs are
    unchanged and the winner is the best kept sample."""
    sc = inputs.tiny_scene(21, 400, 30, 40, width=width, box=30.0, clear=4.0)
    p0 = sc["preset"]
    st = sc["state"].astype(np.float32).astype(np.float64)
    goal_ev, obs_ev = orc.frame_to_ev(st, sc["goal"], sc["obs"])
    z0, ap = [0, 0, 0, st[3]], st[4:6]
    idx = np.arange(400)
    free = orc.rollout_samples(p0, sc["seed"], 2, idx, z0, ap, goal_ev, obs_ev, 30)
    lo, hi = float(st[3]) - 3.0, float(st[3]) + 3.2
    lim = orc.rollout_samples(_limits(p0, lo, hi), sc["seed"], 2, idx, z0, ap, goal_ev, obs_ev, 30)
    v = free["traj"][:, 1:, 3]
    out = (v < lo) | (v > hi)
    hv = np.where(out.any(axis=1), out.argmax(axis=1) + 1, -1)
    fh = free["first_hit"]
    # a speed step counts only while the unconstrained sample is still alive
    hv = np.where((hv >= 0) & ((fh < 0) | (hv < fh)), hv, -1)
    want = np.where(hv >= 0, hv, fh)
    np.testing.assert_array_equal(lim["first_hit"], want)
    kept = want < 0
    assert 20 < kept.sum() < 400 and (hv >= 0).sum() > 100
    np.testing.assert_array_equal(lim["cost"][kept], free["cost"][kept])
    assert np.all(np.isinf(lim["cost"][~kept]))


def test_wide_limits_change_nothing(orc):
    sc = inputs.tiny_scene(22, 64, 25, 80, width=16)
    st = sc["state"].astype(np.float32).astype(np.float64)
    goal_ev, obs_ev = orc.frame_to_ev(st, sc["goal"], sc["obs"])
    a = orc.rollout_samples(sc["preset"], sc["seed"], 1, np.arange(64), [0, 0, 0, st[3]], st[4:6], goal_ev,
                            obs_ev, 25)
    b = orc.rollout_samples(_limits(sc["preset"], -1e6, 1e6), sc["seed"], 1, np.arange(64), [0, 0, 0, st[3]],
                            st[4:6], goal_ev, obs_ev, 25)
    np.testing.assert_array_equal(a["cost"], b["cost"])
    np.testing.assert_array_equal(a["first_hit"], b["first_hit"])


def test_all_discarded_is_infeasible(orc):
    """Limits no sample can meet after one step: every sample is discarded
    at h = 1, the plan reports INFEASIBLE and the lowest index."""
    sc = inputs.tiny_scene(23, 50, 15, 30, width=16)
    p = _limits(sc["preset"], 50.0, 60.0)
    r = orc.plan(p, sc["state"], sc["goal"], sc["obs"], 50, 15, sc["seed"], 0)
    assert r["status"] == 2 and r["best_idx"] == 0
    assert np.all(r["first_hit"] == 1)


def test_body_frame_features_rotate_the_offset(orc):
    p = dict(inputs.planner(16), feature_frame=1)
    pe = inputs.planner(16)
    rng = np.random.default_rng(5)
    for _ in range(20):
        z = np.array([rng.uniform(-20, 20), rng.uniform(-20, 20), rng.uniform(-4, 4), rng.uniform(-3, 10)])
        g = np.array([rng.uniform(-40, 40), rng.uniform(-40, 40), rng.uniform(-3, 3), rng.uniform(0, 5)])
        ap = rng.uniform(-1, 1, 2)
        h, T = int(rng.integers(0, 30)), 30
        sb, se = orc.features(p, z, ap, g, h, T), orc.features(pe, z, ap, g, h, T)
        d = (g[:2] - z[:2]) * np.exp(0j)
        off = complex(d[0], d[1]) * complex(math.cos(-z[2]), math.sin(-z[2]))
        np.testing.assert_allclose([sb[0] * p["dxi_n"], sb[1] * p["deta_n"]], [off.real, off.imag], atol=1e-12)
        np.testing.assert_array_equal(sb[2:], se[2:])
    z = np.array([1.0, 2.0, 0.0, 3.0])
    g = np.array([7.0, -4.0, 0.5, 0.0])
    np.testing.assert_array_equal(orc.features(p, z, [0, 0], g, 0, 10), orc.features(pe, z, [0, 0], g, 0, 10))
    z[2] = math.pi / 2
    s = orc.features(p, z, [0, 0], g, 0, 10)
    np.testing.assert_allclose([s[0] * p["dxi_n"], s[1] * p["deta_n"]], [-6.0, -6.0], atol=1e-12)


def test_body_frame_rollout_first_control_unchanged(orc):
    """At h = 0 the vehicle's heading in the EV frame at t is 0, so the first
    applied control is the EV-frame one; later ones differ once it turns."""
    sc = inputs.tiny_scene(24, 32, 20, 0, width=32)
    st = sc["state"].astype(np.float32).astype(np.float64)
    goal_ev, obs_ev = orc.frame_to_ev(st, sc["goal"], sc["obs"])
    args = (sc["seed"], 0, np.arange(32), [0, 0, 0, st[3]], st[4:6], goal_ev, obs_ev, 20)
    a = orc.rollout_samples(sc["preset"], *args)
    b = orc.rollout_samples(dict(sc["preset"], feature_frame=1), *args)
    np.testing.assert_array_equal(a["ctrl"][:, 0], b["ctrl"][:, 0])
    np.testing.assert_array_equal(a["traj"][:, :2], b["traj"][:, :2])
    assert np.abs(a["ctrl"][:, 5:] - b["ctrl"][:, 5:]).max() > 1e-3
