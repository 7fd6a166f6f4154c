"""Step chunks of the binned plan step: the horizon rolled out in K chunks,
each followed by the check of the states it produced, only the samples
still collision-free going on.  Every output (per-sample costs and first
collisions, the winner, its parameters, rows and controls) must equal the
single launch bit for bit, at every width, with warm starts, the sampling
proposal, speed limits, infeasible scenes and in the closed loop; the work
counters must show exactly the chunk rule (a sample is rolled out through
the chunk holding its first collision and no further)."""
import os
import sys

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


def _planner(sc, chunks, timing=False):
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=max(M, 1))
    npp.npp_set_option(pl.h, "collide_variant", BINNED)
    npp.npp_set_option(pl.h, "fuse", 0)
    npp.npp_set_option(pl.h, "chunks", chunks)
    if timing:
        npp.npp_set_timing(pl.h, True)
    return pl


def _plan(sc, chunks, warm=None, timing=False, proposal=None):
    """One plan step without per-sample records (the chunked path's
    condition); returns the planner's results (and the work counters when
    timing)."""
    import torch
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = _planner(sc, chunks, timing)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda") if M else None
    w = None if warm is None else torch.tensor(warm, dtype=torch.float32, device="cuda")
    if proposal is None:
        pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"], warm=w)
    else:
        mu, sd, n_prop = proposal
        npp.npp_plan_step_proposal(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], sc["t_index"], w,
                                   torch.tensor(mu, device="cuda"), torch.tensor(sd, device="cuda"), n_prop,
                                   pl.outputs())
    torch.cuda.synchronize()
    r = pl.result(N, T)
    if timing:
        r["counts"] = npp.npp_last_counts(pl.h)
        r["timing"] = npp.npp_last_timing(pl.h)
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


def rolled_steps(first_hit, T, K):
    """Sample-steps the chunk rule rolls out: chunk k covers steps
    [T k / K, T (k + 1) / K); a sample takes part in chunk k unless a state
    up to the end of chunk k - 1 collided (its first_hit <= that step)."""
    fh = np.asarray(first_hit)
    total = 0
    for k in range(K):
        lo, hi = T * k // K, T * (k + 1) // K
        prev_end = lo                      # last state checked before chunk k (chunk k - 1 ends at state lo)
        alive = (fh < 0) | (fh > prev_end) if k > 0 else np.ones(fh.shape, bool)
        total += int(alive.sum()) * (hi - lo)
    return total


@pytest.mark.parametrize("width,N,T,M,seed", [(16, 1500, 20, 600, 1), (32, 3000, 33, 1200, 2),
                                              (64, 700, 40, 900, 3), (16, 37, 7, 700, 4)])
@pytest.mark.parametrize("chunks", [2, 3, 5, 8])
def test_chunks_equal_single_launch(width, N, T, M, seed, chunks):
    sc = inputs.tiny_scene(100 + seed, N, T, M, width=width, box=14.0, clear=1.5)
    _assert_same(_plan(sc, chunks), _plan(sc, 1))


def test_chunks_more_than_steps():
    """More chunks asked for than steps: at most one chunk per step."""
    sc = inputs.tiny_scene(110, 800, 3, 700, width=16, box=10.0, clear=1.0)
    one = _plan(sc, 1)
    r = _plan(sc, 8, timing=True)
    _assert_same(r, one)
    assert r["counts"][2] == rolled_steps(one["first_hit"], 3, 3)


def test_chunks_warm_start_and_infeasible():
    """A converging ring of points: every sample collides; the winner (the
    latest first collision) and its rows equal the single launch's, with a
    warm start in sample 0."""
    from paper_1904_06680_gb300 import npp
    p = inputs.planner(32)
    ang = np.linspace(0, 2 * np.pi, 400, endpoint=False)
    obs = np.zeros((400, 4))
    obs[:, 0], obs[:, 1] = 9 * np.cos(ang), 9 * np.sin(ang)
    obs[:, 2], obs[:, 3] = -2 * np.cos(ang), -2 * np.sin(ang)
    sc = dict(preset=p, state=np.array([0.0, 0.0, 0.3, 1.0, 0.1, 0.0]), goal=np.array([6.0, 2.0, 0.0, 0.0]),
              obs=obs, N=2000, T=40, seed=inputs.philox_seed(5), t_index=3)
    warm = (np.random.default_rng(3).standard_normal(1410) * 0.3).astype(np.float32)
    one = _plan(sc, 1, warm=warm)
    assert one["status"] == npp.NPP_INFEASIBLE
    for k in (2, 4, 7):
        _assert_same(_plan(sc, k, warm=warm), one)


def test_chunks_with_proposal():
    """Mixed sampling (proposal samples first, then plain ones)."""
    sc = inputs.tiny_scene(21, N=3000, T=25, M=700, width=16, box=20.0)
    rng = np.random.default_rng(21)
    mu = (rng.standard_normal(450) * 0.5).astype(np.float32)
    sd = np.exp(rng.uniform(-2, 0.5, 450)).astype(np.float32)
    for n_prop in (1000, 3000):
        one = _plan(sc, 1, proposal=(mu, sd, n_prop))
        _assert_same(_plan(sc, 3, proposal=(mu, sd, n_prop)), one)


def test_chunks_with_speed_limits_and_body_frame():
    """Speed limits discard samples like a collision (the first violating
    state joins the first collision); body-frame goal features."""
    sc = inputs.tiny_scene(130, N=2500, T=30, M=800, width=32, box=30.0, clear=4.0)
    v0 = float(np.float32(sc["state"][3]))
    sc = dict(sc, preset=dict(sc["preset"], v_limits=1, v_min=v0 - 3.0, v_max=v0 + 3.2, feature_frame=1))
    one = _plan(sc, 1)
    for k in (2, 4):
        _assert_same(_plan(sc, k), one)


def test_chunk_work_counters_follow_the_chunk_rule():
    """The trajectory launches roll out exactly the chunk rule's
    sample-steps (N T in one launch); the stage times are the chunk sums."""
    sc = inputs.scene_course(0, N=8192)
    N, T = sc["N"], sc["T"]
    one = _plan(sc, 1, timing=True)
    assert one["counts"][2] == N * T
    for k in (2, 4):
        r = _plan(sc, k, timing=True)
        _assert_same(r, one)
        assert r["counts"][2] == rolled_steps(one["first_hit"], T, k)
        assert r["counts"][2] < N * T
        assert r["timing"]["traj"] > 0 and r["timing"]["collide"] > 0
        assert r["timing"]["total"] >= r["timing"]["traj"] + r["timing"]["collide"] - 1e-3


def test_chunks_at_the_large_workload():
    """N = 65536, T = 100, 8-64-64-2, M = 8192: the automatic chunks (2)
    and four chunks against one launch."""
    sc = inputs.scene_large(0)
    one = _plan(sc, 1)
    _assert_same(_plan(sc, 0), one)
    r = _plan(sc, 4, timing=True)
    _assert_same(r, one)
    assert r["counts"][2] == rolled_steps(one["first_hit"], sc["T"], 4)


@pytest.mark.parametrize("restarts", [1, 3])
def test_chunks_in_the_closed_loop(restarts):
    """The graph-captured loop (with and without the hill-climb rounds):
    chunked and single-launch plan steps give the same executed poses, log
    and per-sample results at every sampling time."""
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.scene_course(1, N=4096)
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    obs0 = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    runs = []
    for chunks in (1, 2, 3):
        pl = _planner(sc, chunks)
        npp.npp_set_loop_restarts(pl.h, restarts, 0.1 if restarts > 1 else 0.0)
        L = npp.npp_loop_create(pl.h, sc["state"], sc["waypoints"], inputs.EPS, obs0, M, N, T, sc["seed"])
        samples = []
        for _ in range(6):
            npp.npp_loop_run(L, 1)
            samples.append(npp.npp_loop_samples(L, N))
        runs.append((samples, npp.npp_loop_log(L), npp.npp_loop_read(L)))
        npp.npp_loop_destroy(L)
        pl.close()
    for r in runs[1:]:
        for (c, f), (c0, f0) in zip(r[0], runs[0][0]):
            np.testing.assert_array_equal(f, f0)
            np.testing.assert_array_equal(c.view(np.int32), c0.view(np.int32))
        np.testing.assert_array_equal(r[1], runs[0][1])
        assert r[2] == runs[0][2]


def _plan_fused(sc, variant=0, timing=False):
    """The plan step with the windowed check inside the trajectory kernel
    (option fuse) in launch shape `variant`."""
    import torch
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = _planner(sc, 1, timing)
    npp.npp_set_option(pl.h, "fuse", 1)
    npp.npp_set_option(pl.h, "traj_variant", variant)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda") if M else None
    pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
    torch.cuda.synchronize()
    r = pl.result(N, T)
    if timing:
        r["counts"] = npp.npp_last_counts(pl.h)
    pl.close()
    return r


def window_steps(first_hit, T, CW, per_warp):
    """Control steps the windowed kernel computes: a sample's warp rolls
    windows of CW states until every sample of the warp (per_warp
    consecutive ones) has collided, the window of its first collision
    included; min(CW (k + 1), T) steps through window k."""
    fh = np.asarray(first_hit)
    own = np.where(fh < 0, T, np.minimum((fh // CW + 1) * CW, T))
    pad = (-len(own)) % per_warp
    warp = np.concatenate([own, np.zeros(pad, own.dtype)]).reshape(-1, per_warp).max(axis=1)
    return int(np.repeat(warp, per_warp)[:len(own)].sum())


@pytest.mark.parametrize("width,variants", [(16, (0, 2, 3)), (32, (0, 1, 2, 3, 4)), (64, (0, 1, 2, 3, 4))])
def test_fused_window_shapes_equal_single_launch(width, variants):
    sc = inputs.tiny_scene(140 + width, 2100, 37, 900, width=width, box=14.0, clear=1.5)
    one = _plan(sc, 1)
    for v in variants:
        _assert_same(_plan_fused(sc, v), one)


@pytest.mark.parametrize("width,cw,per_warp", [(64, 8, 1), (32, 8, 2), (16, 16, 4)])
def test_fused_work_counter_follows_the_window_rule(width, cw, per_warp):
    sc = inputs.tiny_scene(150 + width, 3000, 45, 1500, width=width, box=14.0, clear=1.5)
    one = _plan(sc, 1)
    r = _plan_fused(sc, 0, timing=True)
    _assert_same(r, one)
    assert r["counts"][2] == window_steps(one["first_hit"], sc["T"], cw, per_warp)


def test_fused_at_the_large_workload():
    sc = inputs.scene_large(0)
    _assert_same(_plan_fused(sc, 0), _plan(sc, 1))
