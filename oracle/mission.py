"""Plain CPU oracle of the closed-loop mission layer (Alg. 1, Steps 3, 4 and 7;
Sect. II-B to II-D): reference-path indexing, goal setpoint selection within
the range field, stop and completion checks, and the range field's
visibility of obstacle points.  FP64, pure Python loops.

TEST INFRASTRUCTURE ONLY: used by tests/ (and nothing in the product path).

Readings (the paper describes these steps in words only):
* the reference path is a sequence of setpoints (x, y, phi, v); setpoints with
  v = 0 and the last one are stop setpoints (a cusp between forward and
  reverse driving, a parking position) that must be reached within the
  tolerances eps = (xi, eta, phi, v) before the path beyond them is used;
  reaching the last one completes the mission (Sect. II-B);
* the space index tracking progress along the path (Sect. II-C, footnote) is
  the setpoint closest to the vehicle among idx .. min(idx + window, stop),
  ties to the lowest index (it never moves backwards nor past an unreached
  stop);
* the goal setpoint (Sect. II-D (iv)) is the furthest setpoint from the space
  index on, up to the stop, such that it and every setpoint before it lie
  within or on the boundary of the range field, the rectangle
  xi in [-back, front], |eta| <= side in the EV frame at t; the space index
  itself when even that one is outside;
* with hide_outside, obstacle points outside the range field at t are not
  seen by that sampling time's plan step (measurements from the range field
  only, Sect. II-C).
"""
import math


def ev_coords(pose, px, py):
    """(xi, eta) of world point (px, py) in the EV frame of pose (x, y, phi)."""
    c, s = math.cos(pose[2]), math.sin(pose[2])
    dx, dy = px - pose[0], py - pose[1]
    return c * dx + s * dy, -s * dx + c * dy


def in_field(pose, px, py, field):
    """field = (front, back, side); boundary included."""
    xi, eta = ev_coords(pose, px, py)
    return -field[1] <= xi <= field[0] and abs(eta) <= field[2]


def is_stop(ref, k):
    return k == len(ref) - 1 or ref[k][3] == 0.0


def next_stop(ref, k):
    """First stop setpoint at or after k."""
    while not is_stop(ref, k):
        k += 1
    return k


def reached(pose, v, g, eps):
    """Completion tolerances of Table hyperparameters: position error along
    and across the vehicle's heading, heading error (wrapped), speed error."""
    xi, eta = ev_coords(pose, g[0], g[1])
    dphi = math.remainder(g[2] - pose[2], 2.0 * math.pi)
    return abs(xi) <= eps[0] and abs(eta) <= eps[1] and abs(dphi) <= eps[2] and abs(g[3] - v) <= eps[3]


def space_index(ref, pose, idx, stop, window):
    best, bd = idx, math.inf
    for k in range(idx, min(idx + window, stop) + 1):
        d = math.hypot(ref[k][0] - pose[0], ref[k][1] - pose[1])
        if d < bd:
            best, bd = k, d
    return best


def select_goal(ref, pose, idx, stop, field):
    if not in_field(pose, ref[idx][0], ref[idx][1], field):
        return idx
    k = idx
    while k + 1 <= stop and in_field(pose, ref[k + 1][0], ref[k + 1][1], field):
        k += 1
    return k


class Mission:
    """State of the mission layer: space index, next stop, goal index, done."""

    def __init__(self, ref, field, window, eps, pose0):
        self.ref = [tuple(float(v) for v in r) for r in ref]
        self.field = tuple(float(f) for f in field)
        self.window = int(window)
        self.eps = tuple(float(e) for e in eps)
        self.idx = 0
        self.stop = next_stop(self.ref, 0)
        self.done = False
        self.goal = select_goal(self.ref, pose0, self.idx, self.stop, self.field)

    def update(self, pose, v):
        """After the plant moved to (pose, v): Step 7 then Steps 3-4 for the
        next sampling time.  Returns the goal index."""
        if not self.done:
            self.idx = space_index(self.ref, pose, self.idx, self.stop, self.window)
            if reached(pose, v, self.ref[self.stop], self.eps):
                if self.stop == len(self.ref) - 1:
                    self.done = True
                else:
                    self.idx = self.stop
                    self.stop = next_stop(self.ref, self.stop + 1)
            self.goal = select_goal(self.ref, pose, self.idx, self.stop, self.field)
        return self.goal


def visible(points, pose, tau, field):
    """Per obstacle point (x, y, vx, vy) at time tau: inside the range field."""
    return [in_field(pose, p[0] + tau * p[2], p[1] + tau * p[3], field) for p in points]
