"""Pins of the oracle's general footprint (Sect. II-D: the EV as an
arbitrarily refined polytope, convex or non-convex, checked by linear
inequalities): a union of convex pieces with counter-clockwise vertices in
the vehicle's frame.

* The rectangle as a 4-vertex piece against the rectangle check.
* A non-convex L outline (two convex pieces) against an even-odd ray
  casting test of the outline itself, a triangle against barycentric
  coordinates, on dense point grids at random poses.
* Rigid-motion invariance and the margin counts.
* A rollout with a pointed nose against the closed form of a straight run.
"""
import math

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

RECT = [[[-2.25, -0.9], [2.25, -0.9], [2.25, 0.9], [-2.25, 0.9]]]
# L outline (counter-clockwise) and its split into two convex pieces
L_OUTLINE = np.array([[-2.0, -1.0], [2.5, -1.0], [2.5, 0.2], [0.0, 0.2], [0.0, 1.0], [-2.0, 1.0]])
L_PIECES = [[[-2.0, -1.0], [2.5, -1.0], [2.5, 0.2], [-2.0, 0.2]],
            [[-2.0, 0.2], [0.0, 0.2], [0.0, 1.0], [-2.0, 1.0]]]
TRI = [[[-1.0, -1.2], [2.0, 0.0], [-1.0, 1.2]]]


def _ray_cast(poly, q):
    """Even-odd rule: a horizontal ray from q crosses the outline an odd
    number of times iff q is inside."""
    inside = False
    n = len(poly)
    for i in range(n):
        (x0, y0), (x1, y1) = poly[i], poly[(i + 1) % n]
        if (y0 > q[1]) != (y1 > q[1]):
            xc = x0 + (q[1] - y0) * (x1 - x0) / (y1 - y0)
            if q[0] < xc:
                inside = not inside
    return inside


def _barycentric(tri, q):
    (ax, ay), (bx, by), (cx, cy) = tri
    det = (by - cy) * (ax - cx) + (cx - bx) * (ay - cy)
    l1 = ((by - cy) * (q[0] - cx) + (cx - bx) * (q[1] - cy)) / det
    l2 = ((cy - ay) * (q[0] - cx) + (ax - cx) * (q[1] - cy)) / det
    return l1 > 0 and l2 > 0 and 1 - l1 - l2 > 0


def _body(q_world, x, y, phi):
    d = np.asarray(q_world) - [x, y]
    c, s = math.cos(phi), math.sin(phi)
    return np.array([c * d[0] + s * d[1], -s * d[0] + c * d[1]])


def _grid_points(rng, x, y, n=41, half=4.0):
    g = np.linspace(-half, half, n) + rng.uniform(-0.01, 0.01)
    X, Y = np.meshgrid(g + x, g + y)
    return np.stack([X.ravel(), Y.ravel()], 1)


def test_rectangle_piece_equals_rectangle_check(orc):
    p = inputs.planner(16)
    q = dict(p, footprint=RECT)
    rng = np.random.default_rng(0)
    for _ in range(10):
        x, y, phi = rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-4, 4)
        for pt in _grid_points(rng, x, y, n=25):
            o = np.array([[pt[0], pt[1], 0.0, 0.0]])
            assert orc.collide(p, x, y, phi, o)[0] == orc.collide(q, x, y, phi, o)[0]


@pytest.mark.parametrize("pieces,outline,test", [(L_PIECES, L_OUTLINE, _ray_cast), (TRI, np.array(TRI[0]), _barycentric)])
def test_footprint_against_textbook_tests(orc, pieces, outline, test):
    p = dict(inputs.planner(16), footprint=pieces)
    rng = np.random.default_rng(1)
    n_in = 0
    for _ in range(6):
        x, y, phi = rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-4, 4)
        for pt in _grid_points(rng, x, y):
            q = _body(pt, x, y, phi)
            want = test(outline, q)
            got = orc.collide(p, x, y, phi, np.array([[pt[0], pt[1], 0.0, 0.0]]))[0]
            assert got == want, (q, got, want)
            n_in += want
    assert n_in > 100


def test_footprint_rigid_motion_and_velocity(orc):
    """Rotating and translating pose and points together keeps every flag;
    a point moving at constant velocity is checked at p + tau v."""
    p = dict(inputs.planner(16), footprint=L_PIECES)
    rng = np.random.default_rng(2)
    pts = np.zeros((400, 4))
    pts[:, :2] = rng.uniform(-4, 4, (400, 2))
    ang, t = 0.7, np.array([3.0, -8.0])
    c, s = math.cos(ang), math.sin(ang)
    Rm = np.array([[c, -s], [s, c]])
    for phi in (0.0, 1.1, -2.5):
        for k in range(400):
            a = orc.collide(p, 0.2, -0.1, phi, pts[k:k + 1])[0]
            w = pts[k:k + 1].copy()
            w[0, :2] = Rm @ w[0, :2] + t
            xy = Rm @ [0.2, -0.1] + t
            b = orc.collide(p, xy[0], xy[1], phi + ang, w)[0]
            assert a == b
    moving = np.array([[10.0, 0.0, -4.0, 0.0]])          # at tau = 2.4 s it sits at x = 0.4
    assert orc.collide(p, 0, 0, 0, moving, tau=2.4)[0] and not orc.collide(p, 0, 0, 0, moving, tau=1.0)[0]


def test_footprint_margin_counts(orc):
    p = dict(inputs.planner(16), footprint=RECT)
    o = np.array([[0.0, 0.4, 0, 0]])                      # 0.5 m inside the long side
    f, nc, nn = orc.collide(p, 0, 0, 0, o, margin=0.4)
    assert f and nc == 1 and nn == 0
    f, nc, nn = orc.collide(p, 0, 0, 0, o, margin=0.6)
    assert f and nc == 0 and nn == 1
    o = np.array([[0.0, 1.3, 0, 0]])                      # 0.4 m outside
    f, nc, nn = orc.collide(p, 0, 0, 0, o, margin=0.5)
    assert not f and nc == 0 and nn == 1


def test_footprint_rollout_straight_run_closed_form(orc):
    """Constant speed, zero steering (zero network, output biases atanh(a)):
    a point on the centre line X m ahead is first inside a footprint whose
    nose reaches tip m ahead of the reference point at the first h with
    v0 Ts h + tip > X."""
    nose = [[[-2.25, -0.9], [2.0, -0.9], [3.1, 0.0], [2.0, 0.9], [-2.25, 0.9]]]
    p = dict(inputs.planner(16), footprint=nose)
    a1 = -1 - 2 * p["u_min"] / (p["u_max"] - p["u_min"])     # zero acceleration
    nt = orc.n_theta(p)
    th = np.zeros(nt)
    th[-1] = math.atanh(a1)
    v0, X, T = 4.0, 9.03, 30
    r = orc.rollout_theta(p, th[None], [0, 0, 0, v0], [0.0, a1], [50, 0, 0, 4], np.array([[X, 0.0, 0, 0]]), T)
    h = np.arange(T + 1)
    want = int(h[v0 * p["Ts"] * h + 3.1 > X][0])
    assert r["first_hit"][0] == want == 15
    # the rectangle (front at 2.25 m) meets it later
    r0 = orc.rollout_theta(inputs.planner(16), th[None], [0, 0, 0, v0], [0.0, a1], [50, 0, 0, 4],
                           np.array([[X, 0.0, 0, 0]]), T)
    assert r0["first_hit"][0] == int(h[v0 * p["Ts"] * h + 2.25 > X][0]) == 17
