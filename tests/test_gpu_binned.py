"""Per-step spatial binning of the obstacle points (collision variant 5)
against the brute-force check: collision flags, costs and the chosen sample
must be identical, since the binned kernel applies the same per-point test
to a superset of the points that can be inside the vehicle rectangle."""
import math
import sys
import os

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
import parity  # noqa: E402

pytestmark = pytest.mark.gpu

BINNED = 5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(sc, variant, pl=None, fuse=0):
    import torch
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    own = pl is None
    if own:
        pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=max(M, 1))
    npp.npp_set_option(pl.h, "collide_variant", variant)
    npp.npp_set_option(pl.h, "fuse", fuse)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda") if M else None
    pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
    torch.cuda.synchronize()
    r = pl.result(N, T)
    if own:
        pl.close()
    return r


def _assert_same(a, b):
    np.testing.assert_array_equal(a["first_hit"], b["first_hit"])
    np.testing.assert_array_equal(a["costs"].view(np.int32), b["costs"].view(np.int32))
    assert (a["best_idx"], a["status"], a["first_hit_best"]) == (b["best_idx"], b["status"], b["first_hit_best"])
    assert np.float32(a["best_cost"]).view(np.int32) == np.float32(b["best_cost"]).view(np.int32)
    np.testing.assert_array_equal(a["params"], b["params"])
    np.testing.assert_array_equal(a["trajectory"], b["trajectory"])
    np.testing.assert_array_equal(a["controls"], b["controls"])


@pytest.mark.parametrize("seed,N,T,M", [(1, 300, 20, 200), (2, 1000, 33, 1500), (3, 77, 5, 1),
                                        (4, 4096, 40, 5000)])
def test_binned_equals_brute_force_random(seed, N, T, M):
    """The two-kernel binned check and the windowed check inside the
    trajectory kernel (fuse=1) against brute force: every sample's flag and
    cost, the winner and its rows."""
    sc = inputs.tiny_scene(seed, N, T, M, width=32, box=25.0, clear=2.0)
    brute = _plan(sc, 3)
    _assert_same(_plan(sc, BINNED), brute)
    _assert_same(_plan(sc, BINNED, fuse=1), brute)


@pytest.mark.parametrize("width", [16, 64])
def test_fused_binned_other_widths(width):
    sc = inputs.tiny_scene(40 + width, 1500, 30, 900, width=width, box=25.0, clear=2.0)
    brute = _plan(sc, 2)
    _assert_same(_plan(sc, BINNED), brute)
    _assert_same(_plan(sc, BINNED, fuse=1), brute)


def test_fused_infeasible_and_warm_start():
    """All samples collide (a converging ring of points): the windowed
    check reports the latest first collision and the winner's rows repeat
    the colliding state with zero controls after it, as the two-kernel path
    does."""
    import torch
    from paper_1904_06680_gb300 import npp
    p = inputs.planner(32)
    ang = np.linspace(0, 2 * np.pi, 400, endpoint=False)
    obs = np.zeros((400, 4))
    obs[:, 0], obs[:, 1] = 9 * np.cos(ang), 9 * np.sin(ang)
    obs[:, 2], obs[:, 3] = -2 * np.cos(ang), -2 * np.sin(ang)
    sc = dict(preset=p, state=np.array([0.0, 0.0, 0.3, 1.0, 0.1, 0.0]), goal=np.array([6.0, 2.0, 0.0, 0.0]),
              obs=obs, N=2000, T=40, seed=inputs.philox_seed(5), t_index=3)
    from paper_1904_06680_gb300 import npp as _npp
    b = _plan(sc, 2)
    for fuse in (0, 1):
        a = _plan(sc, BINNED, fuse=fuse)
        assert a["status"] == _npp.NPP_INFEASIBLE
        _assert_same(a, b)


@pytest.mark.parametrize("width,N,T,M", [(64, 1, 1, 0), (64, 33, 8, 1), (64, 130, 9, 300), (64, 65, 17, 300),
                                         (16, 1, 7, 300), (16, 33, 16, 300), (16, 130, 17, 0), (32, 3, 9, 50)])
def test_fused_degenerate_sizes(width, N, T, M):
    """The windowed check at the edges of its windows and groups: horizons
    of one step, one window (8 states at width 64, 16 at width 16) and one
    past it, a single sample, sample counts that leave a warp's groups
    partly empty, no points and one point -- bit for bit the brute-force
    check's results."""
    sc = inputs.tiny_scene(200 + N + T, N, T, M, width=width, box=12.0, clear=1.0)
    brute = _plan(sc, 2)
    _assert_same(_plan(sc, BINNED, fuse=1), brute)
    _assert_same(_plan(sc, BINNED), brute)


def test_points_beyond_shared_memory():
    """More points than shared memory holds: the brute-force check reads the
    EV-frame pairs from global memory (written in the staging's blocked
    layout); the same flags and winner as the binned check."""
    sc = inputs.tiny_scene(77, N=600, T=10, M=20000, width=16, box=40.0, clear=1.0)
    brute = _plan(sc, 3)
    assert np.any(brute["first_hit"] >= 0)
    _assert_same(_plan(sc, BINNED), brute)


def test_binned_without_points():
    sc = inputs.tiny_scene(5, 500, 20, 0, width=16)
    r = _plan(sc, BINNED)
    assert np.all(r["first_hit"] == -1)
    _assert_same(r, _plan(sc, 3))


def test_binned_points_on_cell_edges():
    """EV frame = world frame (start at the origin, heading 0, so the frame
    change is exact): points on the grid lines of the binning and one float
    step either side of them, around a fan of slow trajectories."""
    p = inputs.planner(16)
    R = math.sqrt(p["half_len"] ** 2 + p["half_wid"] ** 2) + abs(p["c_off"])
    cell = np.float32(2.0 * R + 0.25)
    x0 = np.float32(-0.5 * 128 * float(cell))
    pts = []
    for k in range(58, 71):
        g = np.float32(x0 + np.float32(k) * cell)
        for x in (np.nextafter(g, np.float32(-1e9)), g, np.nextafter(g, np.float32(1e9))):
            for y in np.linspace(-12, 12, 37, dtype=np.float32):
                pts.append((float(x), float(y)))
                pts.append((float(y), float(x)))
    pts = np.array(pts)
    pts = pts[np.hypot(pts[:, 0], pts[:, 1]) > 2.5]
    obs = np.zeros((len(pts), 4))
    obs[:, :2] = pts
    sc = dict(preset=p, state=np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0]),
              goal=np.array([8.0, 3.0, 0.5, 0.0]), obs=obs, N=2048, T=30,
              seed=inputs.philox_seed(11), t_index=4)
    a, b = _plan(sc, BINNED), _plan(sc, 2)
    assert 0 < np.count_nonzero(a["first_hit"] >= 0) < sc["N"]
    _assert_same(a, b)


def test_binned_beyond_the_grid():
    """Trajectories that leave the binning grid (fast start) and points far
    outside it: both are clamped to the border cells the same way."""
    p = inputs.planner(16)
    rng = np.random.default_rng(9)
    M = 3000
    obs = np.zeros((M, 4))
    obs[:1000, 0] = rng.uniform(300, 420, 1000)           # across the grid border at ~326 m
    obs[:1000, 1] = rng.uniform(-40, 40, 1000)
    obs[1000:2000, :2] = rng.uniform(-5e3, 5e3, (1000, 2))  # far outside
    obs[2000:, 0] = rng.uniform(5, 300, 1000)
    obs[2000:, 1] = rng.choice([-1, 1], 1000) * rng.uniform(3.0, 30.0, 1000)
    obs[2000:2500, 2] = -rng.uniform(0, 5, 500)
    sc = dict(preset=p, state=np.array([0.0, 0.0, 0.0, 95.0, 0.0, 0.0]),
              goal=np.array([400.0, 0.0, 0.0, 95.0]), obs=obs, N=4096, T=40,
              seed=inputs.philox_seed(12), t_index=0)
    a, b = _plan(sc, BINNED), _plan(sc, 2)
    fh = a["first_hit"]
    assert np.any(fh >= 0) and np.any(fh < 0)
    _assert_same(a, b)


def test_binned_large_against_oracle():
    """N = 65536, T = 100, 8-64-64-2, 8192 points: binned plan step, sampled
    collision decisions re-evaluated in FP64 at the GPU's own states, and the
    oracle's free-running rollouts of the same samples."""
    sc = inputs.scene_large(0)
    g = parity.gpu_plan(sc, record=True)
    assert g["status"] == 0
    idx = np.unique(np.concatenate([np.arange(64), np.random.default_rng(0).choice(sc["N"], 192, False),
                                    [g["best_idx"]]]))
    fs = parity.flag_stats(sc, g, idx)
    assert not fs["bad"], fs["bad"][:5]
    assert fs["checked"] > 1000
    o = parity.oracle_samples(sc, idx, record=False)
    agree = np.mean(o["first_hit"] == g["first_hit"][idx])
    assert agree >= 0.9, agree


def test_binned_closed_loop_identical_to_brute_force():
    """20 closed-loop sampling times of the large scene, once with binning and
    once brute force: every step's plan and therefore the whole run are
    identical; the per-sample flags of steps 0 and 19 are compared."""
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.scene_large(0)
    p, N, T = sc["preset"], sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    obs0 = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    runs = {}
    for variant, fuse in ((BINNED, 0), (2, 0), (BINNED, 1)):
        pl = npp.Planner(p, max_N=N, max_T=T, max_M=M)
        npp.npp_set_option(pl.h, "collide_variant", variant)
        npp.npp_set_option(pl.h, "fuse", fuse)
        L = npp.npp_loop_create(pl.h, sc["state"], sc["waypoints"], inputs.EPS, obs0, M, N, T, sc["seed"])
        npp.npp_loop_run(L, 1)
        s0 = npp.npp_loop_samples(L, N)
        npp.npp_loop_run(L, 19)
        s19 = npp.npp_loop_samples(L, N)
        runs[(variant, fuse)] = (s0, s19, npp.npp_loop_log(L), npp.npp_loop_read(L))
        npp.npp_loop_destroy(L)
        pl.close()
    b = runs[(2, 0)]
    for a in (runs[(BINNED, 0)], runs[(BINNED, 1)]):
        for k in range(2):
            np.testing.assert_array_equal(a[k][1], b[k][1])
            np.testing.assert_array_equal(a[k][0].view(np.int32), b[k][0].view(np.int32))
        np.testing.assert_array_equal(a[2], b[2])
        assert a[3] == b[3]
    a = runs[(BINNED, 0)]
    assert a[3]["t"] == 20
    assert np.any(a[1][1] < 0)                # feasible plans at step 19


@pytest.mark.parametrize("N,T,M", [(1, 1, 0), (1, 1, 1), (1, 3, 600), (33, 1, 600), (5, 2, 2)])
def test_all_variants_at_extreme_sizes(N, T, M):
    """One sample, one step, no or one point: every collision variant (brute
    force 0-4, binned in two kernels and windowed) gives the same result."""
    sc = inputs.tiny_scene(60 + N + T + M, N, T, M, width=16, box=6.0, clear=1.0)
    ref = _plan(sc, 2)
    for v in (0, 1, 3, 4):
        _assert_same(_plan(sc, v), ref)
    for fuse in (0, 1):
        _assert_same(_plan(sc, BINNED, fuse=fuse), ref)
