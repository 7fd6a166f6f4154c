"""GPU parity of the general footprint (Sect. II-D: the EV as a refined
polytope, convex or non-convex): a union of convex pieces checked by
strict linear inequalities.

* The binned polygon check against the brute-force polygon check (every
  point each step): identical flags, costs and winner.
* Collision decisions at the GPU's own states re-evaluated by the oracle's
  cross-product test (FP64, 1e-4 m ambiguity margin), per-step replay,
  free-running trajectories and the chosen sample.
* The rectangle given as a polygon against the rectangle kernels.
* Speed limits with a footprint, the closed loop, the full-size course
  scene, and the argument checks.
"""
import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

from . import parity as P

pytestmark = pytest.mark.gpu

RECT = [[[-2.25, -0.9], [2.25, -0.9], [2.25, 0.9], [-2.25, 0.9]]]
# a car with a pointed nose and a tow bar: two convex pieces, non-convex union
CAR = [[[-2.25, -0.9], [1.8, -0.9], [2.6, -0.3], [2.6, 0.3], [1.8, 0.9], [-2.25, 0.9]],
       [[-3.3, -0.1], [-2.2, -0.1], [-2.2, 0.1], [-3.3, 0.1]]]
L_SHAPE = [[[-2.0, -1.0], [2.5, -1.0], [2.5, 0.2], [-2.0, 0.2]],
           [[-2.0, 0.2], [0.0, 0.2], [0.0, 1.0], [-2.0, 1.0]]]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _with(sc, **kw):
    sc = dict(sc)
    sc["preset"] = dict(sc["preset"], **kw)
    return sc


def _plan(sc, variant=-1, record=False):
    import torch
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=max(M, 1), record_samples=record)
    npp.npp_set_option(pl.h, "collide_variant", variant)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda") if M else None
    pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
    torch.cuda.synchronize()
    r = pl.result(N, T)
    pl.close()
    return r


def _same(a, b):
    np.testing.assert_array_equal(a["first_hit"], b["first_hit"])
    np.testing.assert_array_equal(a["costs"].view(np.int32), b["costs"].view(np.int32))
    assert (a["best_idx"], a["status"]) == (b["best_idx"], b["status"])
    np.testing.assert_array_equal(a["trajectory"], b["trajectory"])
    np.testing.assert_array_equal(a["controls"], b["controls"])


@pytest.mark.parametrize("fp", [RECT, CAR, L_SHAPE])
@pytest.mark.parametrize("seed,N,T,M,width,box", [(101, 700, 25, 400, 16, 25.0), (102, 2000, 30, 1500, 32, 60.0),
                                                  (103, 33, 3, 1, 64, 25.0), (104, 257, 12, 0, 16, 25.0)])
def test_binned_polygon_equals_brute_force(fp, seed, N, T, M, width, box):
    sc = _with(inputs.tiny_scene(seed, N=N, T=T, M=M, width=width, box=box, clear=3.0), footprint=fp)
    a, b = _plan(sc, -1), _plan(sc, 2)
    _same(a, b)
    if M > 100:
        assert 0 < np.count_nonzero(a["first_hit"] >= 0) < N


@pytest.mark.parametrize("fp", [CAR, L_SHAPE])
@pytest.mark.parametrize("width,N,T,M,seed", [(16, 300, 20, 60, 111), (32, 150, 24, 90, 112), (64, 70, 18, 40, 113)])
def test_polygon_parity_small(orc, fp, width, N, T, M, seed):
    sc = _with(inputs.tiny_scene(seed, N=N, T=T, M=M, width=width, box=20.0, clear=3.0), footprint=fp)
    g = P.gpu_plan(sc)
    idx = np.arange(N)
    fs = P.flag_stats(sc, g, idx)
    assert not fs["bad"], fs["bad"][:5]
    assert fs["checked"] > N
    rs = P.replay_stats(sc, g, idx)
    assert not rs["bad"], rs["bad"][:5]
    o = P.oracle_samples(sc, idx)
    frac, ok, err, kap, _ = P.traj_check(sc, g, idx, o)
    assert frac >= P.CONSISTENT_FRAC, (frac, err[~ok][:5], kap[~ok][:5])
    assert ok[g["best_idx"]]
    ca = P.cost_at_gpu_states(sc, g, idx)
    assert np.nanmax(ca, initial=0.0) <= P.COST_RTOL, np.nanmax(ca)
    wc = P.winner_check(g, o["cost"], o["first_hit"])
    if not wc.get("infeasible"):
        assert wc["ok"], wc
    assert 0 < np.count_nonzero(g["first_hit"] >= 0) < N


def test_rectangle_polygon_matches_rectangle_kernels():
    """The same rectangle two ways (scaled rows with the sign-bit test, and
    half-planes in the vehicle's frame): decisions differ only where a point
    sits within rounding of a face."""
    sc = inputs.tiny_scene(121, N=4096, T=30, M=2000, width=32, box=60.0, clear=3.0)
    a = _plan(sc)
    b = _plan(_with(sc, footprint=RECT))
    agree = np.mean(a["first_hit"] == b["first_hit"])
    assert agree >= 0.998, agree
    assert 0 < np.count_nonzero(a["first_hit"] >= 0) < sc["N"]


def test_polygon_with_speed_limits():
    sc = inputs.tiny_scene(122, N=1500, T=30, M=300, width=16, box=40.0, clear=4.0)
    v0 = float(np.float32(sc["state"][3]))
    sc = _with(sc, footprint=CAR, v_limits=1, v_min=v0 - 3.0, v_max=v0 + 3.2)
    a, b = _plan(sc, -1), _plan(sc, 2)
    _same(a, b)
    free = _plan(_with(sc, v_limits=0))
    assert np.count_nonzero(a["first_hit"] >= 0) > np.count_nonzero(free["first_hit"] >= 0)
    # every sample kept with limits is kept without them, with the same cost
    kept = a["first_hit"] < 0
    np.testing.assert_array_equal(a["costs"][kept], free["costs"][kept])


def test_polygon_course_full_size(orc):
    """The course workload (N = 16384, T = 40, 2000 points) with the car
    footprint: binned against brute force on every sample, oracle decisions
    at the GPU's states on a sample of indices."""
    sc = _with(inputs.scene_course(0), footprint=CAR)
    a, b = _plan(sc, -1, record=True), _plan(sc, 2)
    for k in ("first_hit", "costs"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["best_idx"] == b["best_idx"]
    idx = np.unique(np.concatenate([np.random.default_rng(3).choice(sc["N"], 200, False), [a["best_idx"]]]))
    fs = P.flag_stats(sc, a, idx)
    assert not fs["bad"], fs["bad"][:5]


def test_polygon_closed_loop_runs():
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.scene_course(0, N=4096)
    p = dict(sc["preset"], footprint=CAR)
    M = sc["obs"].shape[0]
    pl = npp.Planner(p, max_N=sc["N"], max_T=sc["T"], max_M=M)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    L = npp.npp_loop_create(pl.h, sc["state"], sc["waypoints"], inputs.EPS, obs, M, sc["N"], sc["T"], sc["seed"])
    npp.npp_loop_run(L, 15)
    st = npp.npp_loop_read(L)
    costs, fh = npp.npp_loop_samples(L, sc["N"])
    npp.npp_loop_destroy(L)
    pl.close()
    assert st["t"] == 15 and st["n_infeasible"] == 0
    assert 0 < np.count_nonzero(fh < 0) <= sc["N"]


def test_footprint_arguments():
    from paper_1904_06680_gb300 import npp
    p = inputs.planner(16)
    pl = npp.Planner(p, max_N=8, max_T=4, max_M=1)
    bad = [[[[0, 0], [1, 0], [0, 1], [1, 1]]],                     # self-intersecting
           [[[0, 0], [0, 1], [1, 0]]],                               # clockwise
           [[[0, 0], [1, 0]]],                                       # two vertices
           [[[0, 0], [1, 0], [2, 0], [0, 1]]],                       # collinear
           [[[np.nan, 0], [1, 0], [0, 1]]],
           [[[np.cos(a), np.sin(a)] for a in np.arange(5) * 4 * np.pi / 5]],   # pentagram: winds twice
           [RECT[0]] * 17,
           [[[np.cos(a), np.sin(a)] for a in np.linspace(0, 2 * np.pi, 66)[:-1]]]]
    for fp in bad:
        with pytest.raises(npp.NppError):
            npp.npp_set_footprint(pl.h, fp)
    npp.npp_set_footprint(pl.h, CAR)
    scenes = npp.make_scenes([dict(state=[0] * 6, goal=[1, 0, 0, 0], N=8, T=4, M=0, width=16, obs_offset=0,
                                   seed=1, t_index=0)])
    with pytest.raises(npp.NppError):
        npp.npp_batch_create(pl.h, scenes)
    npp.npp_set_footprint(pl.h, [])
    B = npp.npp_batch_create(pl.h, scenes)
    npp.npp_batch_destroy(B)
    pl.close()
