"""Seeded synthetic inputs and configuration presets.

This module holds only configuration values and seeded input generators; it
contains none of the method's arithmetic, so that both the CUDA path and the
CPU oracle can be driven from the same inputs.  Numbers come from the paper's
tables (vehicle constants, Table veh; hyperparameters, Table hyperparameters)
and from the planner workloads this library is benchmarked on.

Scene recipes (all world-frame, SI units; obstacles are (x, y, vx, vy)):

* ``scene_single``: one planning instance, N = 256, T = 20, 8-16-16-2 network,
  200 static points uniform in a 40 x 40 m box centred on the start with none
  within 5 m of it, goal position uniform in the box, goal heading uniform,
  goal speed 0, start at rest with a random world pose.
* ``scene_batch``: S independent reverse-parking instances (the slot of the
  paper's Experiment 5, Fig. 8: curb line, a 5 x 5 m slot and a top wall,
  resampled at 0.25 m and scaled 1.25x for the 4.5 m car), each at a random
  world pose, with N = round(exp U[ln 1024, ln 65536]) rounded up to a
  multiple of 32, T ~ U{20..80}, M = round(exp U[ln 100, ln 20000]) points
  (the walls, parked-car outlines and a boundary wall, and 30 % of the points
  on car outlines moving at |v| <= 3 m/s along a far lane), hidden width
  uniform in {16, 32, 64}; start on the road at rest, goal at rest inside
  the slot facing out.
* ``scene_course``: the forward/reverse waypoint course of the paper's
  Experiment 4 (four waypoints at the corners of a square, heading turned by
  90 degrees at each) scaled 1.5x; 2000 points: 1000 on an outer wall, 500 on
  a central island, 500 on ten moving car-sized outlines with speeds uniform
  in [0, 3] m/s at uniform headings.  N = 16384, T = 40, 8-32-32-2.
* ``scene_large``: N = 65536, T = 100, 8-64-64-2, 8192 points over an
  80 x 80 m area centred on the start: a boundary wall at 0.25 m spacing,
  parked-car outlines at uniform positions and headings (none within 8 m of
  the start or 5 m of the goal), and 20 % of the points on moving car
  outlines with speeds uniform in [0, 5] m/s at uniform headings (none
  starting within 10 m of the start).  Start at the origin at rest facing
  +x; waypoints 30 m out.
* ``scene_proposal_batch``: scenes for training and evaluating the learned
  sampling proposal, shaped like the course workload: each scene uses one of
  `n_layouts` course obstacle layouts (``scene_course`` with its own seed:
  outer wall, island, ten moving car outlines; 2000 points) and a random
  start pose in the free area (heading uniform, speed U[0, 2] m/s, last
  controls U[-0.3, 0.3], no point within 2.5 m) with a goal 6-15 m away in
  a uniform direction, heading within +-90 degrees of the start heading,
  at rest, also clear of points.  8-16-16-2 network, N = 4096, T = 40.
* ``scene_mission``: a transportation mission along a winding two-lane road
  (centre line y = 4 sin(2 pi x / 60), x in [0, 150] m): the reference path
  samples the centre line every 1 m at 4 m/s with the last setpoint at rest;
  both road bounds are points every 0.5 m, 3.5 m either side; six parked-car
  outlines (0.5 m spacing) sit in the lane, one at a random station in each of
  six 20 m slots from x = 20 m (neighbours at least 18 m apart),
  alternately left and right of the centre line (their centre 2.2 m
  off it, aligned with the road); one car outline drives towards the
  vehicle in the far lane at 1 m/s.  Start at rest on the centre line.
  8-32-32-2, N = 8192, T = 40; range field 25 m ahead, 8 m behind, 10 m to
  either side.
* ``scene_turnaround``: the paper's Experiment 1 (Sect. V): start at rest at
  the origin facing +x, one waypoint at the origin facing -x at rest, no
  obstacle points (one point parked 10 km away, so the kernels see M = 1);
  the paper's vehicle (Table veh) with an 8-16-16-2 network, N = 16384,
  T = 80; `seed` picks the sampler's Philox seed.
* ``scene_waypoints``: the paper's Experiment 4 (Sect. V): start at rest at
  the origin, the four waypoints of ``scene_course`` (forward and reverse
  driving with 90-degree heading changes), no obstacle points (one parked
  10 km away); 8-32-32-2, N = 16384, T = 40.
* ``scene_parking``: the reverse parking mission of the paper's Experiment 5
  (Fig. 8, bottom row) in the scaled slot layout of ``scene_batch``: start at
  rest at (0, 2.5) facing +x, an auxiliary waypoint at the origin facing +y,
  then the parking position inside the slot (0, -6.25) facing +y, both at
  rest; the walls as points every 0.25 m; 8-16-16-2, N = 16384, T = 60.
"""
import math

import numpy as np

# ------------------------------------------------------------------ presets
PAPER = dict(
    # Table veh: l_f, l_r, delta_max, delta_dot_max, u_min, u_max
    lf=1.1, lr=1.4, delta_max=40 * math.pi / 180, delta_rate_max=20 * math.pi / 180,
    u_min=-100 / (3.8 * 3.6), u_max=100 / (7.4 * 3.6), Ts=0.1,
    # chassis (l_f + 0.7 + l_r + 0.6) x 2 m around the CoG: 1.8 m ahead,
    # 2.0 m behind -> centre 0.1 m behind the CoG
    half_len=1.9, half_wid=1.0, c_off=-0.1,
    # Table hyperparameters: Delta xi, Delta eta, Delta phi, Delta v
    dxi_n=30.0, deta_n=3.5, dphi_n=2 * math.pi, dv_n=120 / 3.6,
    w_pos=1.0, w_phi=1.0, w_v=0.1, w_effort=0.1,
    widths=(5, 2, 2),
)


def planner(width: int) -> dict:
    """4.5 x 1.8 m car, wheelbase 2.7 m (reference point mid-wheelbase at the
    rectangle centre), steering +-0.6 rad at 20 deg/s, acceleration +-3 m/s^2,
    Ts = 0.1 s, 8-width-width-2 tanh network."""
    return dict(
        lf=1.35, lr=1.35, delta_max=0.6, delta_rate_max=20 * math.pi / 180,
        u_min=-3.0, u_max=3.0, Ts=0.1,
        half_len=2.25, half_wid=0.9, c_off=0.0,
        dxi_n=30.0, deta_n=3.5, dphi_n=2 * math.pi, dv_n=120 / 3.6,
        w_pos=1.0, w_phi=1.0, w_v=0.1, w_effort=0.1,
        widths=(8, width, width, 2),
    )


# paper Table hyperparameters: completion tolerances (xi, eta, phi, v)
EPS = (1.0, 0.25, 10 * math.pi / 180, 5 / 3.6)


def philox_seed(scene_seed: int) -> int:
    return 0x5EED0000 + int(scene_seed)


# ------------------------------------------------------------------ scenes
def scene_single(seed: int = 0, N: int = 256, T: int = 20, M: int = 200, width: int = 16):
    rng = np.random.default_rng(1000 + seed)
    x0, y0 = rng.uniform(-100, 100, 2)
    phi0 = rng.uniform(-math.pi, math.pi)
    pts = []
    while len(pts) < M:
        p = rng.uniform(-20, 20, 2)
        if p[0] ** 2 + p[1] ** 2 >= 25.0:
            pts.append(p)
    pts = np.array(pts).reshape(-1, 2) + [x0, y0]
    obs = np.zeros((M, 4))
    obs[:, :2] = pts
    g = rng.uniform(-20, 20, 2) + [x0, y0]
    goal = np.array([g[0], g[1], rng.uniform(-math.pi, math.pi), 0.0])
    state = np.array([x0, y0, phi0, 0.0, 0.0, 0.0])
    return dict(preset=planner(width), state=state, goal=goal, obs=obs, N=N, T=T,
                seed=philox_seed(seed), t_index=0)


def _square_outline(cx, cy, half_l, half_w, heading, n):
    """n points evenly spaced along a rectangle's perimeter."""
    per = 4 * (half_l + half_w)
    s = (np.arange(n) + 0.5) * per / n
    pts = np.zeros((n, 2))
    for i, d in enumerate(s):
        if d < 2 * half_l:
            pts[i] = (-half_l + d, -half_w)
        elif d < 2 * half_l + 2 * half_w:
            pts[i] = (half_l, -half_w + d - 2 * half_l)
        elif d < 4 * half_l + 2 * half_w:
            pts[i] = (half_l - (d - 2 * half_l - 2 * half_w), half_w)
        else:
            pts[i] = (-half_l, half_w - (d - 4 * half_l - 2 * half_w))
    c, s_ = math.cos(heading), math.sin(heading)
    return np.stack([cx + c * pts[:, 0] - s_ * pts[:, 1], cy + s_ * pts[:, 0] + c * pts[:, 1]], 1)


COURSE_WAYPOINTS = np.array([
    [15.0, 0.0, math.pi / 2, 0.0],
    [15.0, 15.0, math.pi, 0.0],
    [0.0, 15.0, -math.pi / 2, 0.0],
    [0.0, 0.0, 0.0, 0.0],
])


def scene_course(seed: int = 0, N: int = 16384, T: int = 40, width: int = 32,
                 n_wall: int = 1000, n_island: int = 500, n_dyn: int = 500, vmax: float = 3.0):
    rng = np.random.default_rng(2000 + seed)
    wall = _square_outline(7.5, 7.5, 15.5, 15.5, 0.0, n_wall)
    half = n_island // 2
    island = np.concatenate([_square_outline(7.5, 7.5, 2.5, 2.5, 0.0, half),
                             rng.uniform(5.0, 10.0, (n_island - half, 2))])
    n_clusters = max(1, n_dyn // 50)
    dyn = []
    vel = []
    per = [n_dyn // n_clusters + (1 if i < n_dyn % n_clusters else 0) for i in range(n_clusters)]
    for k in range(n_clusters):
        while True:
            c = rng.uniform(-6.0, 21.0, 2)
            if np.hypot(*c) > 8.0 and not (3.0 < c[0] < 12.0 and 3.0 < c[1] < 12.0):
                break
        hd = rng.uniform(-math.pi, math.pi)
        speed = rng.uniform(0.0, vmax)
        vh = rng.uniform(-math.pi, math.pi)
        dyn.append(_square_outline(c[0], c[1], 2.25, 0.9, hd, per[k]))
        vel.append(np.tile([speed * math.cos(vh), speed * math.sin(vh)], (per[k], 1)))
    dyn = np.concatenate(dyn)
    vel = np.concatenate(vel)
    obs = np.zeros((n_wall + n_island + n_dyn, 4))
    obs[:n_wall, :2] = wall
    obs[n_wall:n_wall + n_island, :2] = island
    obs[n_wall + n_island:, :2] = dyn
    obs[n_wall + n_island:, 2:] = vel
    state = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    return dict(preset=planner(width), state=state, goal=COURSE_WAYPOINTS[0].copy(), obs=obs,
                N=N, T=T, seed=philox_seed(seed), t_index=0, waypoints=COURSE_WAYPOINTS.copy())


LARGE_WAYPOINTS = np.array([
    [30.0, 8.0, 0.0, 0.0],
    [30.0, 30.0, math.pi / 2, 0.0],
])


def scene_large(seed: int = 0, N: int = 65536, T: int = 100, width: int = 64, M: int = 8192,
                dyn_frac: float = 0.2, vmax: float = 5.0, n_parked: int = 50, area: float = 80.0):
    rng = np.random.default_rng(5000 + seed)
    half = area / 2
    n_dyn = int(round(dyn_frac * M))
    n_static = M - n_dyn
    wall = _square_outline(0.0, 0.0, half, half, 0.0, min(n_static // 4, int(round(4 * area / 0.25))))
    rest = n_static - len(wall)
    per = [rest // n_parked + (1 if i < rest % n_parked else 0) for i in range(n_parked)]
    goal = LARGE_WAYPOINTS[0]
    parked = []
    for k in range(n_parked):
        while True:
            c = rng.uniform(-half + 3.0, half - 3.0, 2)
            if np.hypot(*c) > 8.0 and np.hypot(c[0] - goal[0], c[1] - goal[1]) > 5.0:
                break
        parked.append(_square_outline(c[0], c[1], 2.25, 0.9, rng.uniform(-math.pi, math.pi), per[k]))
    n_mov = max(1, n_dyn // 100)
    perm = [n_dyn // n_mov + (1 if i < n_dyn % n_mov else 0) for i in range(n_mov)]
    dyn, vel = [], []
    for k in range(n_mov):
        while True:
            c = rng.uniform(-half + 3.0, half - 3.0, 2)
            if np.hypot(*c) > 10.0:
                break
        sp = rng.uniform(0.0, vmax)
        vh = rng.uniform(-math.pi, math.pi)
        dyn.append(_square_outline(c[0], c[1], 2.25, 0.9, rng.uniform(-math.pi, math.pi), perm[k]))
        vel.append(np.tile([sp * math.cos(vh), sp * math.sin(vh)], (perm[k], 1)))
    obs = np.zeros((M, 4))
    obs[:n_static, :2] = np.concatenate([wall] + parked)
    obs[n_static:, :2] = np.concatenate(dyn)
    obs[n_static:, 2:] = np.concatenate(vel)
    state = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    return dict(preset=planner(width), state=state, goal=goal.copy(), obs=obs, N=N, T=T,
                seed=philox_seed(seed), t_index=0, waypoints=LARGE_WAYPOINTS.copy())


def scene_proposal_batch(seed: int = 0, S: int = 512, N: int = 4096, T: int = 40, n_layouts: int = 16):
    rng = np.random.default_rng(6000 + seed)
    layouts = [scene_course(seed=10000 + 97 * seed + l)["obs"] for l in range(n_layouts)]
    M = layouts[0].shape[0]
    scenes = []

    def clear(obs, x, y):
        return np.min(np.hypot(obs[:, 0] - x, obs[:, 1] - y)) > 2.5

    for s_ in range(S):
        l = s_ % n_layouts
        obs = layouts[l]
        while True:
            x, y = rng.uniform(-5.0, 20.0, 2)
            if not (2.0 < x < 13.0 and 2.0 < y < 13.0) and clear(obs, x, y):
                break
        phi = rng.uniform(-math.pi, math.pi)
        while True:
            d = rng.uniform(6.0, 15.0)
            a = phi + rng.uniform(-math.pi, math.pi)
            gx, gy = x + d * math.cos(a), y + d * math.sin(a)
            if -5.0 < gx < 20.0 and -5.0 < gy < 20.0 and not (2.0 < gx < 13.0 and 2.0 < gy < 13.0) \
                    and clear(obs, gx, gy):
                break
        gphi = phi + rng.uniform(-math.pi / 2, math.pi / 2)
        state = np.array([x, y, phi, rng.uniform(0.0, 2.0), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)])
        goal = np.array([gx, gy, gphi, 0.0])
        scenes.append(dict(state=state, goal=goal, N=N, T=T, M=M, width=16, obs_offset=l * M,
                           seed=philox_seed(seed) * 1000003 + s_, t_index=0))
    return dict(preset=planner(16), scenes=scenes, obs=np.concatenate(layouts))


def tiny_scene(seed: int, N: int, T: int, M: int, width: int = 16, box: float = 12.0,
               dyn_frac: float = 0.3, vmax: float = 3.0, clear: float = 3.0):
    """Small random instance for exhaustive checks: M points uniform in a
    box around a random start pose (none within `clear` m of it), a fraction
    moving, a random goal, random start speed and last controls."""
    rng = np.random.default_rng(3000 + seed)
    x0, y0 = rng.uniform(-30, 30, 2)
    phi0 = rng.uniform(-math.pi, math.pi)
    pts = []
    while len(pts) < M:
        p = rng.uniform(-box, box, 2)
        if np.hypot(*p) >= clear:
            pts.append(p)
    obs = np.zeros((M, 4))
    if M:
        obs[:, :2] = np.array(pts) + [x0, y0]
        nd = int(round(dyn_frac * M))
        sp = rng.uniform(0, vmax, nd)
        hd = rng.uniform(-math.pi, math.pi, nd)
        obs[:nd, 2] = sp * np.cos(hd)
        obs[:nd, 3] = sp * np.sin(hd)
    g = rng.uniform(-box, box, 2) + [x0, y0]
    goal = np.array([g[0], g[1], rng.uniform(-math.pi, math.pi), rng.uniform(-2, 2)])
    state = np.array([x0, y0, phi0, rng.uniform(-3, 3), rng.uniform(-1, 1), rng.uniform(-1, 1)])
    return dict(preset=planner(width), state=state, goal=goal, obs=obs, N=N, T=T,
                seed=philox_seed(seed), t_index=int(rng.integers(0, 1000)))


def _segment(a, b, spacing):
    n = max(2, int(round(np.hypot(b[0] - a[0], b[1] - a[1]) / spacing)) + 1)
    return np.stack([np.linspace(a[0], b[0], n), np.linspace(a[1], b[1], n)], 1)


def parking_walls(scale: float = 1.25, spacing: float = 0.25) -> np.ndarray:
    """Wall points of the Experiment 5 layout (curb y = -2 for |x| in
    [2.5, 6.5], slot sides x = +-2.5 and bottom y = -7, top wall y = 6 for
    |x| <= 4), resampled and scaled."""
    segs = [((-6.5, -2), (-2.5, -2)), ((-2.5, -2), (-2.5, -7)), ((-2.5, -7), (2.5, -7)),
            ((2.5, -7), (2.5, -2)), ((2.5, -2), (6.5, -2)), ((-4, 6), (4, 6))]
    pts = [_segment(np.array(a) * scale, np.array(b) * scale, spacing) for a, b in segs]
    return np.unique(np.round(np.concatenate(pts), 6), axis=0)


def _car_outline(cx, cy, heading, spacing):
    n = max(8, int(round(2 * (4.5 + 1.8) / spacing)))
    return _square_outline(cx, cy, 2.25, 0.9, heading, n)


def scene_batch(seed: int = 0, S: int = 512, width_choices=(16, 32, 64), N_range=(1024, 65536),
                T_range=(20, 80), M_range=(100, 20000), dyn_frac: float = 0.3, vmax: float = 3.0):
    """See the module docstring.  Points beyond the slot walls are structure,
    not noise: parked-car outlines in rows left and right of the slot and
    beyond the top wall, a boundary wall 30 m out, and (the moving 30 %) car
    outlines driving along a far lane 10-14 m above the road; the road
    between the curb and the top wall and the slot itself stay free.  Large
    M densifies the outlines (smaller point spacing)."""
    rng = np.random.default_rng(4000 + seed)
    walls = parking_walls()
    start_l = np.array([0.0, 2.0 * 1.25, 0.0])
    goal_l = np.array([0.0, -5.0 * 1.25, math.pi / 2])
    slots_x = [x for x in np.arange(-22.5, 23.0, 3.0) if abs(x) > 5.0]
    scenes = []
    obs_chunks = []
    off = 0
    for s in range(S):
        N = int(round(math.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1])))))
        N = max(32, 32 * ((N + 31) // 32))
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        M = int(round(math.exp(rng.uniform(math.log(M_range[0]), math.log(M_range[1])))))
        M = max(M, 1)
        width = int(width_choices[rng.integers(0, len(width_choices))])
        n_dyn = int(round(dyn_frac * M))
        n_static = M - n_dyn
        # static structure: slot walls first, then parked cars and boundary
        # wall sharing the rest; densify until the count is reached
        static = [walls]
        rest = n_static - len(walls)
        if rest > 0:
            n_cars = len(slots_x) * 2
            per_car = max(8, rest // (2 * n_cars))
            spacing = 2 * (4.5 + 1.8) / per_car
            cars = []
            for x in slots_x:
                cars.append(_car_outline(x, -4.6, math.pi / 2, spacing))      # along the curb
                cars.append(_car_outline(x, 9.0, math.pi / 2, spacing))       # beyond the top wall
            cars = np.concatenate(cars)
            nb = max(0, rest - len(cars))
            bound = _square_outline(0.0, 0.0, 30.0, 30.0, 0.0, max(nb, 4))
            static += [cars, bound]
        static = np.concatenate(static)
        if len(static) >= n_static:
            static = static[rng.permutation(len(static))[:n_static]] if n_static > len(walls) else walls[:n_static]
        # moving car outlines on a far lane
        dyn = np.zeros((0, 2))
        dvel = np.zeros((0, 2))
        if n_dyn:
            n_mov = max(1, n_dyn // 60)
            per = [n_dyn // n_mov + (1 if i < n_dyn % n_mov else 0) for i in range(n_mov)]
            chunks, vels = [], []
            for k in range(n_mov):
                cx = rng.uniform(-25, 25)
                cy = rng.uniform(11.0, 13.0)
                sp = rng.uniform(0, vmax) * (1 if rng.random() < 0.5 else -1)
                chunks.append(_square_outline(cx, cy, 2.25, 0.9, 0.0, per[k]))
                vels.append(np.tile([sp, 0.0], (per[k], 1)))
            dyn = np.concatenate(chunks)
            dvel = np.concatenate(vels)
        loc = np.concatenate([static, dyn])[:M]
        vel = np.concatenate([np.zeros((len(static), 2)), dvel])[:M]
        # random rigid placement of the layout in the world
        ang = rng.uniform(-math.pi, math.pi)
        tx, ty = rng.uniform(-500, 500, 2)
        c, sn = math.cos(ang), math.sin(ang)
        R = np.array([[c, -sn], [sn, c]])
        obs = np.zeros((len(loc), 4))
        obs[:, :2] = loc @ R.T + [tx, ty]
        obs[:, 2:] = vel @ R.T
        st = np.concatenate([R @ start_l[:2] + [tx, ty], [start_l[2] + ang, 0.0, 0.0, 0.0]])
        gl = np.concatenate([R @ goal_l[:2] + [tx, ty], [goal_l[2] + ang, 0.0]])
        scenes.append(dict(state=st, goal=gl, N=N, T=T, M=len(loc), width=width, obs_offset=off,
                           seed=philox_seed(seed) + 7919 * s, t_index=0))
        obs_chunks.append(obs)
        off += len(loc)
    return dict(preset=planner(32), scenes=scenes, obs=np.concatenate(obs_chunks))


# a general footprint (vehicle frame, counter-clockwise pieces): a car body
# with a pointed nose and a tow bar behind it; the union is not convex
CAR_FOOTPRINT = [
    [[-2.25, -0.9], [1.8, -0.9], [2.6, -0.3], [2.6, 0.3], [1.8, 0.9], [-2.25, 0.9]],
    [[-3.3, -0.1], [-2.2, -0.1], [-2.2, 0.1], [-3.3, 0.1]],
]

# ------------------------------------------------------------------ missions
MISSION_FIELD = (25.0, 8.0, 10.0)       # range field: front, back, side [m]


def _road(x):
    y = 4.0 * np.sin(2 * math.pi * x / 60.0)
    dy = 4.0 * 2 * math.pi / 60.0 * np.cos(2 * math.pi * x / 60.0)
    return y, np.arctan(dy)


def scene_mission(seed: int = 0, N: int = 8192, T: int = 40, width: int = 32, length: float = 150.0,
                  n_parked: int = 6, lane_speed: float = 4.0):
    """See the module docstring."""
    rng = np.random.default_rng(6000 + seed)
    xs = np.arange(0.0, length + 0.5, 1.0)
    ys, hs = _road(xs)
    ref = np.stack([xs, ys, hs, np.full_like(xs, lane_speed)], 1)
    ref[-1, 3] = 0.0
    xb = np.arange(-10.0, length + 10.0, 0.5)
    yb, hb = _road(xb)
    nx, ny = -np.sin(hb), np.cos(hb)
    bounds = np.concatenate([np.stack([xb + 3.5 * nx, yb + 3.5 * ny], 1),
                             np.stack([xb - 3.5 * nx, yb - 3.5 * ny], 1)])
    # one station per slot of equal length, placed so that neighbours are at
    # least 18 m apart
    slot = (length - 30.0) / n_parked
    stations = [20.0 + k * slot + rng.uniform(0.0, max(slot - 18.0, 0.0)) for k in range(n_parked)]
    cars = []
    side = 1.0 if rng.uniform() < 0.5 else -1.0
    for c in stations:
        yc, hc = _road(np.array([c]))
        cars.append(_square_outline(c - side * 2.2 * math.sin(hc[0]), yc[0] + side * 2.2 * math.cos(hc[0]),
                                    2.25, 0.9, hc[0], 25))
        side = -side
    xo = length - 20.0
    yo, ho = _road(np.array([xo]))
    oncoming = _square_outline(xo - 1.75 * math.sin(ho[0]), yo[0] + 1.75 * math.cos(ho[0]), 2.25, 0.9,
                               ho[0], 25)
    static = np.concatenate([bounds] + cars)
    obs = np.zeros((len(static) + len(oncoming), 4))
    obs[:len(static), :2] = static
    obs[len(static):, :2] = oncoming
    obs[len(static):, 2] = -1.0
    state = np.array([0.0, ref[0, 1], ref[0, 2], 0.0, 0.0, 0.0])
    return dict(preset=planner(width), state=state, goal=ref[-1].copy(), obs=obs, N=N, T=T,
                seed=philox_seed(seed), t_index=0, ref=ref, field=MISSION_FIELD, window=20)


def scene_parking(seed: int = 0, N: int = 16384, T: int = 60, width: int = 16):
    """See the module docstring (the scene is fixed; `seed` picks the
    sampler's Philox seed, as the paper's ten random seeds)."""
    walls = parking_walls()
    obs = np.zeros((len(walls), 4))
    obs[:, :2] = walls
    waypoints = np.array([[0.0, 0.0, math.pi / 2, 0.0], [0.0, -6.25, math.pi / 2, 0.0]])
    state = np.array([0.0, 2.5, 0.0, 0.0, 0.0, 0.0])
    return dict(preset=planner(width), state=state, goal=waypoints[0].copy(), obs=obs, N=N, T=T,
                seed=philox_seed(seed), t_index=0, waypoints=waypoints)


def scene_turnaround(seed: int = 0, N: int = 16384, T: int = 80):
    """See the module docstring (Experiment 1)."""
    obs = np.array([[1e4, 1e4, 0.0, 0.0]])
    waypoints = np.array([[0.0, 0.0, math.pi, 0.0]])
    return dict(preset=dict(PAPER, widths=(8, 16, 16, 2)), state=np.zeros(6), goal=waypoints[0].copy(), obs=obs,
                N=N, T=T, seed=philox_seed(seed), t_index=0, waypoints=waypoints)


def scene_paper_road(with_points: bool = True, seed: int = 0, N: int = 20480, T: int = 200):
    """The paper's Step-5 setting on a road (Experiments 2 and 3, Sect. V):
    the paper's vehicle on this library's smallest network (8-16-16-2), start
    at 50 km/h, goal 60 m ahead at the same speed, horizon H = 200; with
    points: 16 road bounds (every 10 m from 5 to 75 m at +-3.5 m) and 4 on
    the corners of a car 30 m ahead moving at 20 km/h (20 points), else one
    point 10 km away."""
    v0 = 50 / 3.6
    if with_points:
        obs = np.zeros((20, 4))
        obs[:16, 0] = np.tile(np.linspace(5.0, 75.0, 8), 2)
        obs[:16, 1] = np.repeat([-3.5, 3.5], 8)
        obs[16:, 0] = [29.0, 29.0, 33.5, 33.5]
        obs[16:, 1] = [-0.9, 0.9, -0.9, 0.9]
        obs[16:, 2] = 20 / 3.6
    else:
        obs = np.array([[1e4, 1e4, 0.0, 0.0]])
    return dict(preset=dict(PAPER, widths=(8, 16, 16, 2)), state=np.array([0.0, 0.0, 0.0, v0, 0.0, 0.0]),
                goal=np.array([60.0, 0.0, 0.0, v0]), obs=obs, N=N, T=T, seed=philox_seed(seed), t_index=0)


def scene_waypoints(seed: int = 0, N: int = 16384, T: int = 40):
    """See the module docstring (Experiment 4)."""
    obs = np.array([[1e4, 1e4, 0.0, 0.0]])
    return dict(preset=planner(32), state=np.zeros(6), goal=COURSE_WAYPOINTS[0].copy(), obs=obs, N=N, T=T,
                seed=philox_seed(seed), t_index=0, waypoints=COURSE_WAYPOINTS.copy())
