"""The seeded workload generators produce the stated shapes, sizes and value
distributions (CPU only)."""
import math

import numpy as np

from paper_1904_06680_gb300 import inputs


def test_scene_single_recipe():
    sc = inputs.scene_single(3)
    o, s = sc["obs"], sc["state"]
    assert o.shape == (200, 4) and sc["N"] == 256 and sc["T"] == 20
    d = o[:, :2] - s[:2]
    assert np.all(np.abs(d) <= 20.0) and np.all(np.hypot(d[:, 0], d[:, 1]) >= 5.0)
    assert np.all(o[:, 2:] == 0.0)
    assert sc["preset"]["widths"] == (8, 16, 16, 2)


def test_scene_course_recipe():
    sc = inputs.scene_course(1)
    o = sc["obs"]
    assert o.shape == (2000, 4) and sc["N"] == 16384 and sc["T"] == 40
    moving = np.hypot(o[:, 2], o[:, 3])
    assert np.all(moving[:1500] == 0.0) and np.all(moving <= 3.0 + 1e-12)
    assert len(sc["waypoints"]) == 4


def test_scene_large_recipe():
    sc = inputs.scene_large(2)
    o = sc["obs"]
    assert o.shape == (8192, 4) and sc["N"] == 65536 and sc["T"] == 100
    assert sc["preset"]["widths"] == (8, 64, 64, 2)
    speed = np.hypot(o[:, 2], o[:, 3])
    n_dyn = int(np.count_nonzero(np.any(o[:, 2:] != 0.0, axis=1)))
    assert abs(n_dyn - round(0.2 * 8192)) <= 20
    assert np.all(speed <= 5.0 + 1e-12)
    assert np.all(np.abs(o[:, :2]) <= 40.0 + 1e-9)
    static = speed == 0.0
    r = np.hypot(o[:, 0], o[:, 1])
    assert np.min(r[static]) > 8.0 - 2.5          # parked outlines centred beyond 8 m
    assert np.min(r[~static]) > 10.0 - 2.5


def test_scene_batch_recipe():
    b = inputs.scene_batch(0, S=24)
    assert len(b["scenes"]) == 24
    off = 0
    for s in b["scenes"]:
        assert s["obs_offset"] == off
        off += s["M"]
        assert 1024 <= s["N"] <= 65536 + 31 and s["N"] % 32 == 0
        assert 20 <= s["T"] <= 80 and 1 <= s["M"] <= 20000
        assert s["width"] in (16, 32, 64)
        seg = b["obs"][s["obs_offset"]:s["obs_offset"] + s["M"]]
        assert np.all(np.hypot(seg[:, 2], seg[:, 3]) <= 3.0 + 1e-9)
        g, st = s["goal"], s["state"]
        assert math.hypot(g[0] - st[0], g[1] - st[1]) < 15.0
    assert off == b["obs"].shape[0]


def test_mission_scenes_generate_with_spaced_cars():
    """Every seed builds (no rejection loop) with the parked cars at least
    18 m apart along the road and the reference path ending at rest."""
    import time
    t0 = time.perf_counter()
    for seed in range(50):
        sc = inputs.scene_mission(seed)
        assert sc["ref"][-1, 3] == 0.0 and np.all(sc["ref"][:-1, 3] > 0)
        cars = sc["obs"][1 + 2 * len(np.arange(-10.0, 160.0, 0.5)) - 1:-25, :2]
        xs = np.sort(cars.reshape(6, 25, 2)[:, :, 0].mean(axis=1))
        # centres sit 2.2 m off the centre line: along x they move by <= 2.2 sin(0.41) each
        assert np.all(np.diff(xs) >= 18.0 - 2 * 2.2 * 0.4), (seed, xs)
    assert time.perf_counter() - t0 < 5.0


def test_paper_experiment_scenes():
    """Experiment 1 (turn-around) and 4 (four waypoints) as the paper sets
    them up (Sect. V): start at rest at the origin, no obstacle points (one
    point parked 10 km away), goals at rest."""
    import math
    e1 = inputs.scene_turnaround(3)
    assert np.array_equal(e1["state"], np.zeros(6))
    assert np.allclose(e1["waypoints"], [[0.0, 0.0, math.pi, 0.0]])
    assert e1["obs"].shape == (1, 4) and np.min(np.hypot(e1["obs"][:, 0], e1["obs"][:, 1])) > 1e3
    assert e1["preset"]["widths"] == (8, 16, 16, 2) and e1["preset"]["lf"] == inputs.PAPER["lf"]
    e4 = inputs.scene_waypoints(3)
    assert np.array_equal(e4["state"], np.zeros(6)) and e4["waypoints"].shape == (4, 4)
    assert np.all(e4["waypoints"][:, 3] == 0.0)
    assert e1["seed"] != inputs.scene_turnaround(4)["seed"]


def test_scene_paper_road_recipe():
    """The paper's Step-5 road: its vehicle, 50 km/h, goal 60 m ahead, H = 200;
    16 static road bounds at +-3.5 m and a car's 4 corners moving at 20 km/h,
    or a single far point."""
    sc = inputs.scene_paper_road(True)
    o = sc["obs"]
    assert o.shape == (20, 4) and sc["N"] == 20480 and sc["T"] == 200
    assert sc["preset"]["lf"] == inputs.PAPER["lf"] and sc["preset"]["widths"] == (8, 16, 16, 2)
    assert math.isclose(sc["state"][3], 50 / 3.6) and sc["goal"][0] == 60.0
    assert np.all(np.abs(o[:16, 1]) == 3.5) and np.all(o[:16, 2:] == 0.0)
    assert np.allclose(o[16:, 2], 20 / 3.6) and np.all(o[16:, 3] == 0.0) and np.all(np.abs(o[16:, 1]) < 1.0)
    empty = inputs.scene_paper_road(False, N=4096)
    assert empty["obs"].shape == (1, 4) and np.hypot(*empty["obs"][0, :2]) > 1e3 and empty["N"] == 4096
