"""Closed-loop driver around the plan step (Alg. 1 of the paper).

Per sampling time t: the current world-frame state and obstacle points are
the measurements (Step 3), the current waypoint is the goal setpoint
(Step 4, waypoint sequencing only), the library plans (Step 5), the first
applied control of the winner drives the simulated vehicle for one sampling
time (Step 6), the waypoint advances once it is reached within the
tolerances of Table hyperparameters (Step 7), and the winner's parameters
warm-start the next plan (Sect. II-D "Fifth").  The simulated vehicle is the
same kinematic bicycle (Sect. IV) integrated in FP64 on the host; obstacle
points move at their constant velocities.
"""
import math

import numpy as np


def plant_step(p: dict, state: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Advance the simulated vehicle by one sampling time with applied
    normalised controls a = (a0, a1); returns the new 6-vector
    (x, y, phi, v, a_prev0, a_prev1)."""
    x, y, phi, v = state[:4]
    L = p["lf"] + p["lr"]
    delta = p["delta_max"] * a[0]
    u = p["u_min"] + 0.5 * (a[1] + 1.0) * (p["u_max"] - p["u_min"])
    beta = math.atan(p["lr"] * math.tan(delta) / L)
    Ts = p["Ts"]
    return np.array([x + Ts * v * math.cos(phi + beta) / math.cos(beta),
                     y + Ts * v * math.sin(phi + beta) / math.cos(beta),
                     phi + Ts * v * math.tan(delta) / L,
                     v + Ts * u, a[0], a[1]])


def advance_obstacles(obs: np.ndarray, Ts: float) -> np.ndarray:
    out = obs.copy()
    out[:, :2] += Ts * obs[:, 2:]
    return out


def reached(state: np.ndarray, goal: np.ndarray, eps) -> bool:
    """Goal pose within (eps_xi, eps_eta, eps_phi, eps_v) of the vehicle,
    position error measured along and across the vehicle heading."""
    c, s = math.cos(state[2]), math.sin(state[2])
    dx, dy = goal[0] - state[0], goal[1] - state[1]
    dxi, deta = c * dx + s * dy, -s * dx + c * dy
    dphi = math.remainder(goal[2] - state[2], 2 * math.pi)
    return (abs(dxi) <= eps[0] and abs(deta) <= eps[1] and abs(dphi) <= eps[2]
            and abs(goal[3] - state[3]) <= eps[3])


class Mission:
    """Waypoint sequence with completion check."""

    def __init__(self, waypoints: np.ndarray, eps):
        self.waypoints = np.asarray(waypoints, dtype=np.float64)
        self.eps = eps
        self.k = 0

    @property
    def goal(self) -> np.ndarray:
        return self.waypoints[min(self.k, len(self.waypoints) - 1)]

    @property
    def done(self) -> bool:
        return self.k >= len(self.waypoints)

    def update(self, state: np.ndarray) -> None:
        if not self.done and reached(state, self.goal, self.eps):
            self.k += 1
