"""Pins of the mission-layer oracle (Alg. 1 Steps 3, 4, 7): space index,
goal selection within the range field, stop setpoints, completion and the
range field's visibility of points, on paths whose answers follow from the
geometry by hand."""
import math

import numpy as np

from oracle import mission as MS

EPS = (1.0, 0.25, 10 * math.pi / 180, 5 / 3.6)


def _straight(n=61, v=2.0):
    ref = [(float(k), 0.0, 0.0, v) for k in range(n)]
    ref[-1] = (float(n - 1), 0.0, 0.0, 0.0)
    return ref


def _cusp():
    """Forward along x to a stop at x = 20, then reverse back to x = 0."""
    fwd = [(float(k), 0.0, 0.0, 2.0) for k in range(20)] + [(20.0, 0.0, 0.0, 0.0)]
    rev = [(20.0 - k, 0.0, 0.0, -2.0) for k in range(1, 20)] + [(0.0, 0.0, 0.0, 0.0)]
    return fwd + rev


def test_goal_on_the_field_boundary():
    ref = _straight()
    pose = (0.0, 0.0, 0.0)
    assert MS.select_goal(ref, pose, 0, 60, (10.0, 5.0, 3.0)) == 10       # x = 10 on the front edge
    assert MS.select_goal(ref, pose, 0, 60, (9.5, 5.0, 3.0)) == 9
    assert MS.select_goal(ref, pose, 0, 60, (200.0, 5.0, 3.0)) == 60      # the final setpoint
    assert MS.select_goal(ref, pose, 0, 25, (200.0, 5.0, 3.0)) == 25      # never past the stop
    # heading 90 deg: the path runs across the vehicle, |eta| > side beyond x = 3
    assert MS.select_goal(ref, (0.0, 0.0, math.pi / 2), 0, 60, (10.0, 5.0, 3.0)) == 3
    # the space index itself outside the field: the goal is the space index
    assert MS.select_goal(ref, (30.0, 0.0, 0.0), 12, 60, (10.0, 5.0, 3.0)) == 12


def test_lateral_edge_of_a_bending_path():
    ref = [(float(k), 0.25 * k * k, 0.0, 2.0) for k in range(10)] + [(10.0, 25.0, 0.0, 0.0)]
    # eta_k = k^2 / 4 <= 3  <=>  k <= 3
    assert MS.select_goal(ref, (0.0, 0.0, 0.0), 0, 10, (50.0, 5.0, 3.0)) == 3


def test_space_index_window_and_barrier():
    ref = _straight()
    assert MS.space_index(ref, (17.4, 0.3, 0.0), 0, 60, 40) == 17
    assert MS.space_index(ref, (17.5, 0.0, 0.0), 0, 60, 40) == 17          # tie -> lowest index
    assert MS.space_index(ref, (17.4, 0.3, 0.0), 0, 60, 5) == 5
    assert MS.space_index(ref, (17.4, 0.3, 0.0), 0, 12, 40) == 12          # not past the stop
    assert MS.space_index(ref, (3.0, 0.0, 0.0), 8, 60, 10) == 8            # never backwards


def test_cusp_and_completion():
    ref = _cusp()
    assert MS.next_stop(ref, 0) == 20 and MS.next_stop(ref, 21) == 40 and MS.is_stop(ref, 40)
    m = MS.Mission(ref, (50.0, 5.0, 3.0), 30, EPS, (0.0, 0.0, 0.0))
    assert (m.idx, m.stop, m.goal) == (0, 20, 20)
    m.update((10.2, 0.1, 0.0), 2.0)
    assert (m.idx, m.stop, m.goal) == (10, 20, 20)
    m.update((19.5, 0.0, 0.0), 1.5)               # not reached: |v - 0| > 5/3.6
    assert (m.idx, m.stop) == (19, 20)            # equidistant from 19 and 20: the lower
    m.update((19.5, 0.0, 0.0), 0.2)               # reached within the tolerances
    assert (m.idx, m.stop) == (20, 40)
    # reverse segment: setpoints behind the vehicle, back = 5 reaches x = 14.5
    assert m.goal == 25
    m.update((0.4, 0.1, 0.05), -0.3)
    assert m.done and m.goal == 40
    g = m.update((5.0, 0.0, 0.0), 3.0)            # done: nothing changes
    assert g == 40 and m.done


def test_reached_tolerances():
    g = (10.0, 5.0, 0.3, 1.0)
    pose = (10.0 - 0.9 * math.cos(0.3), 5.0 - 0.9 * math.sin(0.3), 0.3)     # 0.9 m behind along the heading
    assert MS.reached(pose, 1.0, g, EPS)
    pose2 = (pose[0] - 0.3 * math.sin(0.3), pose[1] + 0.3 * math.cos(0.3), 0.3)   # 0.3 m to the side
    assert not MS.reached(pose2, 1.0, g, EPS)
    assert not MS.reached((10.0, 5.0, 0.3 + 0.2), 1.0, g, EPS)
    assert MS.reached((10.0, 5.0, 0.3 + 2 * math.pi), 1.0, g, EPS)          # wrapped heading
    assert not MS.reached((10.0, 5.0, 0.3), 1.0 + 1.5, g, EPS)


def test_visibility_of_points():
    pts = [(5.0, 0.0, 0.0, 0.0), (5.0, 3.5, 0.0, 0.0), (-6.0, 0.0, 0.0, 0.0), (20.0, 0.0, -5.0, 0.0),
           (0.0, 10.0, 0.0, 0.0)]
    pose = (0.0, 0.0, 0.0)
    assert MS.visible(pts, pose, 0.0, (10.0, 5.0, 3.0)) == [True, False, False, False, False]
    assert MS.visible(pts, pose, 2.0, (10.0, 5.0, 3.0)) == [True, False, False, True, False]
    # the same field turned with the vehicle: +y is straight ahead
    assert MS.visible(pts, (0.0, 0.0, math.pi / 2), 0.0, (10.0, 5.0, 3.0)) == [False, False, False, False, True]


def test_mission_replay_invariants():
    """Driving along the cusp path: the index never decreases, the goal lies
    between the index and the stop, and the mission completes."""
    ref = _cusp()
    m = MS.Mission(ref, (8.0, 4.0, 3.0), 10, EPS, (0.0, 0.0, 0.0))
    xs = list(np.linspace(0, 19.8, 60)) + [19.8] * 3 + list(np.linspace(19.8, 0.2, 60))
    vs = [2.0] * 60 + [0.0] * 3 + [-2.0] * 59 + [0.0]
    last = 0
    for x, v in zip(xs, vs):
        m.update((x, 0.0, 0.0), v)
        assert m.idx >= last and m.idx <= m.goal <= m.stop
        last = m.idx
    assert m.done
