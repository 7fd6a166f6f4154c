"""Pins of the proposal oracle (CPU): BF16 rounding against an independent
implementation, the polar histogram against hand-placed points and rigid
motion, the network's gradients against finite differences, the NLL's
stationary point, Adam's first steps in closed form, and the mixed sampler's
reductions to the plain one."""
import math

import numpy as np
import pytest

from oracle import proposal as P
from paper_1904_06680_gb300 import inputs


def test_bf16_rounding_cases():
    cases = {1.0: 1.0, 1.0 + 2 ** -8: 1.0, 1.0 + 3 * 2 ** -8: 1.0 + 2 ** -6,
             1.0 + 2 ** -7: 1.0 + 2 ** -7, -2.5: -2.5, 3.14159265: 3.140625, 0.0: 0.0,
             1.0 + 2 ** -8 + 2 ** -20: 1.0 + 2 ** -7}
    for x, want in cases.items():
        assert P.bf16(x) == want, (x, P.bf16(x), want)


def test_bf16_matches_torch_on_float32_inputs():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(P.bf16(x.astype(np.float64)), t)


def test_polar_hist_hand_placed_points():
    width = 2 * math.pi / 64
    pts = []
    want = np.zeros(64)
    for k, d in [(0, 1.0), (5, 10.0), (32, 19.0), (63, 4.0), (40, 25.0), (5, 2.0)]:
        a = -math.pi + (k + 0.5) * width
        pts.append([d * math.cos(a), d * math.sin(a), 0.0, 0.0])
        want[k] += max(0.0, 1.0 - d / 20.0)
    h, amb = P.polar_hist(np.array(pts))
    np.testing.assert_allclose(h, want, atol=1e-12)
    assert np.all(amb == 0)
    # a point exactly on the +x axis sits on the boundary between bins 31 and 32
    h2, amb2 = P.polar_hist(np.array([[5.0, 0.0, 0, 0]]))
    assert h2[32] == 0.75 and amb2[31] == 0.75 and amb2[32] == 0.75


def test_encoding_rigid_motion_invariant():
    p = inputs.planner(16)
    sc = inputs.tiny_scene(3, 16, 20, 300, box=25.0)
    x0, h0, _ = P.encode(p, sc["state"], sc["goal"], sc["obs"], 20)
    ang, tx, ty = 1.234, -40.0, 17.5
    c, s = math.cos(ang), math.sin(ang)
    Rm = np.array([[c, -s], [s, c]])
    st = sc["state"].copy()
    st[:2] = Rm @ st[:2] + [tx, ty]
    st[2] += ang
    gl = sc["goal"].copy()
    gl[:2] = Rm @ gl[:2] + [tx, ty]
    gl[2] += ang
    ob = sc["obs"].copy()
    ob[:, :2] = ob[:, :2] @ Rm.T + [tx, ty]
    ob[:, 2:] = ob[:, 2:] @ Rm.T
    x1, h1, _ = P.encode(p, st, gl, ob, 20)
    np.testing.assert_allclose(h1, h0, atol=1e-9)
    np.testing.assert_allclose(x1, x0, atol=1e-9)
    assert x0.shape == (72,) and np.all((x0[:64] >= 0) & (x0[:64] < 1))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = P.init_params(3, out_scale=0.5)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.standard_normal(params[k].shape) * 0.1
    X = rng.standard_normal((5, P.N_IN))
    theta = rng.standard_normal((5, P.N_THETA))
    cache = P.forward(params, X, quantize=False)
    g = P.backward(params, cache, theta, quantize=False)
    eps = 1e-6
    for k, idxs in [("W1", [(0, 0), (17, 71), (255, 30)]), ("b1", [(3,), (200,)]),
                    ("W2", [(1, 2), (100, 200)]), ("b2", [(7,)]), ("W3", [(0, 5), (449, 1), (450, 3), (899, 255)]),
                    ("b3", [(10,), (460,), (899,)])]:
        for ix in idxs:
            pp = {kk: vv.copy() for kk, vv in params.items()}
            pp[k][ix] += eps
            lp = P.nll(P.forward(pp, X, quantize=False), theta)
            pp[k][ix] -= 2 * eps
            lm = P.nll(P.forward(pp, X, quantize=False), theta)
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k][ix]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, ix, fd, g[k][ix])


def test_nll_stationary_in_log_std():
    """d/d(ls) [ls + r^2 e^{-2 ls} / 2] = 0 at ls = log |r|: with W3 = 0 the
    network's output is its bias, so set it there and the log-std gradient
    vanishes while the mean gradient is -r e^{-2 ls} / (B n)."""
    params = P.init_params(0)
    params["W3"][:] = 0.0
    theta = np.full((2, P.N_THETA), 0.6)
    params["b3"][:P.N_THETA] = 0.1
    params["b3"][P.N_THETA:] = math.log(0.5)
    X = np.random.default_rng(2).standard_normal((2, P.N_IN))
    c = P.forward(params, X, quantize=False)
    np.testing.assert_allclose(c["mu"], 0.1)
    g = P.backward(params, c, theta, quantize=False)
    assert np.max(np.abs(g["b3"][P.N_THETA:])) < 1e-15
    np.testing.assert_allclose(g["b3"][:P.N_THETA], -0.5 / 0.25 / P.N_THETA, rtol=1e-12)


def test_relu_network_homogeneous():
    params = P.init_params(5, out_scale=1.0)
    X = np.random.default_rng(3).standard_normal((4, P.N_IN))
    y1 = P.forward(params, X, quantize=False)["Y"]
    y2 = P.forward(params, 2.5 * X, quantize=False)["Y"]
    np.testing.assert_allclose(y2, 2.5 * y1, rtol=1e-12, atol=1e-12)


def test_adam_first_steps_closed_form():
    params = P.init_params(0)
    rng = np.random.default_rng(4)
    grads = {k: rng.standard_normal(v.shape) for k, v in params.items()}
    st = P.adam_init()
    lr = 1e-3
    p1, st = P.adam_step(params, grads, st, lr)
    g = P.pack(grads)
    want = P.pack(params) - lr * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(P.pack(p1), want, rtol=0, atol=1e-15)
    p2, st = P.adam_step(p1, grads, st, lr)       # constant gradient: same step again
    np.testing.assert_allclose(P.pack(p2), want - lr * g / (np.abs(g) + 1e-8), atol=1e-14)


def test_mixed_sampler_reductions(orc):
    p = inputs.planner(16)
    sc = inputs.tiny_scene(9, 64, 15, 40, width=16)
    st = sc["state"].astype(np.float32).astype(np.float64)
    goal_ev, obs_ev = orc.frame_to_ev(st, sc["goal"], sc["obs"])
    z0, ap = [0, 0, 0, st[3]], st[4:6]
    idx = np.arange(12)
    nt = orc.n_theta(p)
    # mean 0, std 1: the proposal samples are the stream-1 isotropic samples
    a = orc.rollout_samples(p, sc["seed"], 3, idx, z0, ap, goal_ev, obs_ev, 15, mu=np.zeros(nt),
                            sigma=np.ones(nt), n_prop=12)
    b = orc.rollout_samples(p, sc["seed"], 3, idx, z0, ap, goal_ev, obs_ev, 15, stream=1)
    np.testing.assert_array_equal(a["cost"], b["cost"])
    np.testing.assert_array_equal(a["traj"], b["traj"])
    # std 0: every proposal sample is the mean itself
    mu = orc.theta(sc["seed"], 77, 5, nt).astype(np.float32)
    c = orc.rollout_samples(p, sc["seed"], 3, idx, z0, ap, goal_ev, obs_ev, 15, mu=mu,
                            sigma=np.zeros(nt), n_prop=6)
    d = orc.rollout_theta(p, np.tile(mu.astype(np.float64), (6, 1)), z0, ap, goal_ev, obs_ev, 15)
    np.testing.assert_array_equal(c["cost"][:6], d["cost"])
    # samples at or beyond n_prop are the plain stream-0 samples
    e = orc.rollout_samples(p, sc["seed"], 3, idx, z0, ap, goal_ev, obs_ev, 15)
    np.testing.assert_array_equal(c["cost"][6:], e["cost"][6:])


def test_theta_mixed_reductions(orc):
    nt = 450
    a = orc.theta_mixed(77, 3, 5, nt, np.zeros(nt), np.ones(nt), 6)
    np.testing.assert_array_equal(a, orc.theta(77, 3, 5, nt, stream=1))
    b = orc.theta_mixed(77, 3, 6, nt, np.zeros(nt), np.ones(nt), 6)
    np.testing.assert_array_equal(b, orc.theta(77, 3, 6, nt, stream=0))
    mu = np.linspace(-1, 1, nt).astype(np.float32)
    c = orc.theta_mixed(77, 3, 0, nt, mu, np.zeros(nt), 1)
    np.testing.assert_array_equal(c, mu)
