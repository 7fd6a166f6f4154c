"""Pins for the oracle's vehicle model, control mapping and MLP.

* The Fig. 3 state table (Experiment 1) replayed step by step through the
  oracle's Euler step with the paper's vehicle constants (Table veh).
* Closed forms of the Euler recurrence: straight line for zero steering and
  chords of a circle for constant steering at constant speed, driven through
  the full rollout by a network whose weights are zero.
* Parameter counts of the paper's networks (Table ex2) and the parameter
  layout against numpy matmul.
"""
import math
import os

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig3_states.txt")


def _half_unit(a):
    """half a unit in the 6th significant digit (the print precision)."""
    a = abs(float(a))
    if a == 0.0:
        return 0.0
    return 0.5 * 10.0 ** (math.floor(math.log10(a)) - 5)


def test_fig3_replay(orc):
    """Each printed state z_{k+1} follows from the printed z_k by one Euler
    step of the kinematic bicycle (Sect. IV, Table veh) evaluated on the old
    state, with the acceleration implied by the printed speeds and steering
    on the 2-degree grid that the 20 deg/s rate limit produces at Ts = 0.1 s.

    Error budget: every printed value carries half a unit in its 6th
    significant digit (SI units, phi in rad in [0, 2 pi)); the steering is
    estimated from the printed heading change, so its uncertainty sigma_delta
    follows from the heading and speed print precision and is propagated into
    the position tolerance.  Where the speed is above 1 m/s the steering
    estimate is sharp and must sit on the grid."""
    p = dict(inputs.PAPER)
    d = np.loadtxt(GOLDEN)
    t, X, Y, PHI, V = d[:, 0], d[:, 1], d[:, 2], np.deg2rad(d[:, 3]), d[:, 4] / 3.6
    assert len(t) == 117 and np.allclose(np.diff(t), 0.1)
    L = p["lf"] + p["lr"]
    Ts = p["Ts"]
    step = p["delta_rate_max"] * Ts                 # 2 degrees in rad
    assert abs(math.degrees(step) - 2.0) < 1e-12
    n_checked = n_grid = n_fast = 0
    prev = None
    for k in range(116):
        u = (V[k + 1] - V[k]) / Ts
        a1 = 2 * (u - p["u_min"]) / (p["u_max"] - p["u_min"]) - 1
        hv, hv1 = _half_unit(V[k]), _half_unit(V[k + 1])
        tol_a1 = 2 * (hv + hv1) / Ts / (p["u_max"] - p["u_min"])
        assert -1 - tol_a1 <= a1 <= 1 + tol_a1, (k, u)
        if abs(V[k]) < 1e-9:
            # at rest nothing moves and the steering is not observable
            assert X[k + 1] == X[k] and Y[k + 1] == Y[k]
            continue
        hp, hp1 = _half_unit(PHI[k]), _half_unit(PHI[k + 1])
        dphi = math.remainder(PHI[k + 1] - PHI[k], 2 * math.pi)
        tan_est = dphi * L / (V[k] * Ts)
        delta_est = math.atan(tan_est)
        sig_tan = (hp + hp1) * L / (abs(V[k]) * Ts) + abs(tan_est) * hv / abs(V[k])
        sig_delta = sig_tan * math.cos(delta_est) ** 2
        delta = step * round(delta_est / step)
        assert abs(delta) <= p["delta_max"] + 1e-12
        on_grid = abs(delta_est - delta) <= 3 * sig_delta + 1e-9
        if abs(V[k]) > 1.0:
            n_fast += 1
            assert on_grid, (k, math.degrees(delta_est))
        if on_grid:
            n_grid += 1
            if prev is not None:
                assert abs(delta - prev) <= step + 1e-12, (k, delta, prev)
            prev = delta
        else:
            delta = delta_est
            prev = None
        a0 = delta / p["delta_max"]
        zn = orc.euler_step(p, [X[k], Y[k], PHI[k], V[k]], [a0, a1])
        beta = math.atan(p["lr"] * math.tan(delta) / L)
        chord = Ts * abs(V[k]) / math.cos(beta)
        dbeta = (p["lr"] / L) / math.cos(delta) ** 2 / (1 + math.tan(beta) ** 2)
        spread = Ts * hv / math.cos(beta) + chord * (hp + dbeta * 3 * sig_delta)
        tol_x = _half_unit(X[k]) + _half_unit(X[k + 1]) + spread + 1e-12
        tol_y = _half_unit(Y[k]) + _half_unit(Y[k + 1]) + spread + 1e-12
        assert abs(zn[0] - X[k + 1]) <= tol_x, (k, zn[0], X[k + 1], tol_x)
        assert abs(zn[1] - Y[k + 1]) <= tol_y, (k, zn[1], Y[k + 1], tol_y)
        if on_grid:
            tol_p = hp + hp1 + Ts * hv * abs(math.tan(delta)) / L + 1e-12
            assert abs(math.remainder(zn[2] - PHI[k + 1], 2 * math.pi)) <= tol_p, (k,)
        assert abs(zn[3] - V[k + 1]) <= hv + hv1 + 1e-12
        n_checked += 1
    assert n_checked == 115
    assert n_fast >= 70 and n_grid >= 110, (n_fast, n_grid)


def test_fig3_replay_rejects_wrong_constants(orc):
    """The replay is sensitive to the model: swapping l_f and l_r, or moving
    along the new heading instead of the old one, misses the printed state."""
    p = dict(inputs.PAPER)
    d = np.loadtxt(GOLDEN)
    X, Y, PHI, V = d[:, 1], d[:, 2], np.deg2rad(d[:, 3]), d[:, 4] / 3.6
    k = 50                                   # full left lock, 5+ m/s
    delta = -40.0
    a0 = math.radians(delta) / p["delta_max"]
    a1 = 2 * ((V[k + 1] - V[k]) / 0.1 - p["u_min"]) / (p["u_max"] - p["u_min"]) - 1
    good = orc.euler_step(p, [X[k], Y[k], PHI[k], V[k]], [a0, a1])
    assert abs(good[1] - Y[k + 1]) < 1e-4
    q = dict(p, lf=p["lr"], lr=p["lf"])
    bad = orc.euler_step(q, [X[k], Y[k], PHI[k], V[k]], [a0, a1])
    assert abs(bad[1] - Y[k + 1]) > 1e-2 or abs(bad[0] - X[k + 1]) > 1e-2
    # the same chord taken along the new heading (a semi-implicit step)
    L = p["lf"] + p["lr"]
    beta = math.atan(p["lr"] * math.tan(math.radians(delta)) / L)
    ang = PHI[k + 1] + beta
    xs = X[k] + 0.1 * V[k] * math.cos(ang) / math.cos(beta)
    ys = Y[k] + 0.1 * V[k] * math.sin(ang) / math.cos(beta)
    assert max(abs(xs - X[k + 1]), abs(ys - Y[k + 1])) > 1e-2


def _zero_net_theta(p, a0, a1):
    """all weights and hidden biases zero: the output is (a0, a1) exactly when
    the output biases are atanh(a0), atanh(a1)."""
    nt = sum(o * i + o for i, o in zip(p["widths"][:-1], p["widths"][1:]))
    th = np.zeros(nt)
    th[-2] = math.atanh(a0)
    th[-1] = math.atanh(a1)
    return th


@pytest.mark.parametrize("v0,a1", [(0.0, 0.5), (2.0, -0.3), (-1.5, 1.0 - 1e-9)])
def test_straight_line_closed_form(orc, v0, a1):
    """Zero steering: x_h = Ts (h v0 + u Ts h (h-1)/2), y = phi = 0,
    v_h = v0 + h Ts u, through features -> MLP -> controls -> Euler."""
    p = inputs.planner(16)
    T = 30
    th = _zero_net_theta(p, 0.0, a1)
    r = orc.rollout_theta(p, th[None], [0, 0, 0, v0], [0.0, a1], [50, 3, 1, 0], np.zeros((0, 4)), T)
    u = p["u_min"] + 0.5 * (a1 + 1) * (p["u_max"] - p["u_min"])
    h = np.arange(T + 1)
    Ts = p["Ts"]
    x = Ts * (h * v0 + u * Ts * h * (h - 1) / 2)
    traj = r["traj"][0]
    assert r["first_hit"][0] == -1
    np.testing.assert_allclose(traj[:, 0], x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 1], 0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 2], 0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 3], v0 + h * Ts * u, atol=1e-12)
    np.testing.assert_allclose(r["ctrl"][0], np.tile([0.0, a1], (T, 1)), atol=1e-12)


@pytest.mark.parametrize("a0,v0", [(0.5, 3.0), (-1.0 + 1e-12, 2.0), (0.2, -1.0)])
def test_circle_closed_form(orc, a0, v0):
    """Constant steering at constant speed (u = 0): the Euler points are
    p_k = p_0 + l e^{i(phi0+beta)} (1 - e^{ik dphi}) / (1 - e^{i dphi}) with
    chord l = v Ts / cos(beta), dphi = v Ts tan(delta) / L."""
    p = inputs.planner(32)
    T = 60
    a1 = -1 - 2 * p["u_min"] / (p["u_max"] - p["u_min"])    # zero acceleration
    th = _zero_net_theta(p, a0, a1)
    r = orc.rollout_theta(p, th[None], [0, 0, 0, v0], [a0, a1], [10, 10, 0, 0], np.zeros((0, 4)), T)
    L = p["lf"] + p["lr"]
    delta = p["delta_max"] * a0
    beta = math.atan(p["lr"] * math.tan(delta) / L)
    ell = v0 * p["Ts"] / math.cos(beta)
    dphi = v0 * p["Ts"] * math.tan(delta) / L
    k = np.arange(T + 1)
    w = ell * np.exp(1j * beta) * (1 - np.exp(1j * k * dphi)) / (1 - np.exp(1j * dphi))
    traj = r["traj"][0]
    np.testing.assert_allclose(traj[:, 0], w.real, atol=1e-10)
    np.testing.assert_allclose(traj[:, 1], w.imag, atol=1e-10)
    np.testing.assert_allclose(traj[:, 2], k * dphi, atol=1e-12)
    np.testing.assert_allclose(traj[:, 3], v0, atol=1e-12)
    # the points lie on one circle
    R = abs(ell / (2 * math.sin(dphi / 2)))
    centre = ell * np.exp(1j * beta) / (1 - np.exp(1j * dphi))
    np.testing.assert_allclose(np.abs(traj[:, 0] + 1j * traj[:, 1] - centre), R, rtol=1e-9)


def test_steering_rate_limit(orc):
    """The applied steering moves by at most delta_rate_max Ts / delta_max
    per step and stays in [-1, 1] (Table veh; Figs. 3 and 8 show the
    normalised steering moving in steps of 2/40 = 0.05); acceleration
    commands pass unchanged."""
    p = dict(inputs.PAPER)
    r = p["delta_rate_max"] * p["Ts"] / p["delta_max"]
    assert abs(r - 0.05) < 1e-12
    np.testing.assert_allclose(orc.controls(p, [1.0, -0.7], [0.0, 0.3]), [0.05, -0.7])
    np.testing.assert_allclose(orc.controls(p, [-1.0, 0.2], [0.0, 0.0]), [-0.05, 0.2])
    np.testing.assert_allclose(orc.controls(p, [0.99, 0.0], [0.98, 0.0]), [0.99, 0.0])
    np.testing.assert_allclose(orc.controls(p, [1.0, 0.0], [0.97, 0.0]), [1.0, 0.0])
    np.testing.assert_allclose(orc.controls(p, [-1.0, 0.0], [-0.999, 0.0]), [-1.0, 0.0])


def test_paper_parameter_counts(orc):
    """|theta| of the paper's networks (Table ex2) and of the 8-input ones."""
    for widths, n in [((5, 2, 2), 18), ((5, 10, 2), 82), ((5, 10, 10, 2), 192),
                      ((8, 16, 16, 2), 450), ((8, 32, 32, 2), 1410), ((8, 64, 64, 2), 4866)]:
        assert orc.n_theta(dict(inputs.PAPER, widths=widths)) == n


@pytest.mark.parametrize("widths", [(8, 16, 16, 2), (5, 10, 2), (8, 64, 64, 2)])
def test_mlp_layout_vs_matmul(orc, widths):
    """Per layer W[out][in] row-major then b[out]; tanh on every layer."""
    p = dict(inputs.planner(16), widths=widths)
    rng = np.random.default_rng(4)
    nt = orc.n_theta(p)
    th = rng.standard_normal(nt)
    s = rng.uniform(-1, 1, widths[0])
    x = s
    off = 0
    for i, o in zip(widths[:-1], widths[1:]):
        W = th[off: off + o * i].reshape(o, i)
        b = th[off + o * i: off + o * i + o]
        off += o * i + o
        x = np.tanh(W @ x + b)
    np.testing.assert_allclose(orc.mlp(p, th, s), x, rtol=1e-13, atol=1e-14)


def test_features_worked_example(orc):
    """Eq. (eq_def_stph) on hand-worked numbers: goal 30 m ahead and 3.5 m
    to the right, heading error 3 pi / 2 (wrapped to -pi / 2), speed error
    -120/3.6 m/s, last steering 0.25; project entries: last acceleration
    command, normalised speed, remaining-horizon fraction."""
    p = inputs.planner(16)
    z = [1.0, 2.0, 0.25, 40 / 3.6]
    goal = [31.0, -1.5, 0.25 + 1.5 * math.pi, -80 / 3.6]
    s = orc.features(p, z, [0.25, -0.5], goal, 5, 20)
    np.testing.assert_allclose(s, [1.0, -1.0, -0.25, -1.0, 0.25, -0.5, 1.0 / 3.0, 0.75], atol=1e-14)
    s5 = orc.features(dict(inputs.PAPER), z, [0.25, -0.5], goal, 5, 20)
    assert len(s5) == 5
    np.testing.assert_allclose(s5, [1.0, -1.0, -0.25, -1.0, 0.25], atol=1e-14)
