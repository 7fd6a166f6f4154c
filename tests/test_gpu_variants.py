"""GPU parity of the two rollout variants of Sect. V: velocity constraints by
discarding samples (npp_config.v_limits) and goal offsets in the body frame
at t+h (npp_config.feature_frame = 1).

* Body frame: the small-instance checks of the plain path (every step of
  every sample replayed through the oracle, collision decisions at the GPU's
  own states, free-running trajectories, the chosen sample).
* Speed limits: each sample's discard step re-derived at the GPU's own
  states (first h >= 1 whose FP32 speed is outside the limits, or first
  collision re-evaluated in FP64); every collision kernel, the fused check,
  the batch path and the allocation-free entry point give identical
  results; the closed loop keeps the plant's speed within the limits.
"""
import math

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

from . import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _with(sc, **kw):
    sc = dict(sc)
    sc["preset"] = dict(sc["preset"], **kw)
    return sc


def _speed_scene(seed, N, T, M, width, lo_d=-3.0, hi_d=3.2, box=30.0):
    sc = inputs.tiny_scene(seed, N=N, T=T, M=M, width=width, box=box, clear=4.0)
    v0 = float(np.float32(sc["state"][3]))
    return _with(sc, v_limits=1, v_min=v0 + lo_d, v_max=v0 + hi_d)


def _plan(sc, variant=-1, fuse=0, record=True):
    import torch
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=max(M, 1), record_samples=record)
    npp.npp_set_option(pl.h, "collide_variant", variant)
    npp.npp_set_option(pl.h, "fuse", fuse)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda") if M else None
    pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
    torch.cuda.synchronize()
    r = pl.result(N, T)
    pl.close()
    return r


@pytest.mark.parametrize("width,N,T,M,seed", [(16, 300, 20, 40, 71), (32, 150, 24, 60, 72), (64, 70, 18, 33, 73)])
def test_body_frame_parity_small(orc, width, N, T, M, seed):
    sc = _with(inputs.tiny_scene(seed, N=N, T=T, M=M, width=width), feature_frame=1)
    g = P.gpu_plan(sc)
    idx = np.arange(N)
    rs = P.replay_stats(sc, g, idx)
    assert not rs["bad"], rs["bad"][:5]
    assert rs["steps"] > N
    fs = P.flag_stats(sc, g, idx)
    assert not fs["bad"], fs["bad"][:5]
    o = P.oracle_samples(sc, idx)
    frac, ok, err, kap, _ = P.traj_check(sc, g, idx, o)
    assert frac >= P.CONSISTENT_FRAC, (frac, err[~ok][:5], kap[~ok][:5])
    assert ok[g["best_idx"]]
    ca = P.cost_at_gpu_states(sc, g, idx)
    assert np.nanmax(ca, initial=0.0) <= P.COST_RTOL, np.nanmax(ca)
    wc = P.winner_check(g, o["cost"], o["first_hit"])
    if not wc.get("infeasible"):
        assert wc["ok"], wc
    # the frame matters: the plain path picks other controls
    g0 = P.gpu_plan(_with(sc, feature_frame=0))
    assert not np.array_equal(g0["sample_ctrl"], g["sample_ctrl"])
    np.testing.assert_array_equal(g0["sample_ctrl"][0], g["sample_ctrl"][0])   # phi = 0 at h = 0


def _discard_at_own_states(orc, sc, g, n):
    """(expected discard step, ambiguous) from the GPU's own states of n."""
    p = sc["preset"]
    T = sc["T"]
    _, _, _, _, obs_ev = P.oracle_inputs(sc)
    lo, hi = np.float32(p["v_min"]), np.float32(p["v_max"])
    for h in range(T + 1):
        z = g["sample_traj"][h, n]
        if h > 0 and not (lo <= z[3] <= hi):          # FP32 compare, as the kernel
            return h, False
        flag, n_clear, n_near = orc.collide(p, float(z[0]), float(z[1]), float(z[2]), obs_ev,
                                            tau=h * p["Ts"], margin=P.FACE_MARGIN)
        if n_clear == 0 and n_near > 0:
            return None, True
        if flag:
            return h, False
    return -1, False


@pytest.mark.parametrize("width,N,T,M,seed", [(16, 400, 30, 40, 81), (32, 333, 25, 120, 82), (64, 97, 20, 60, 83)])
def test_speed_limits_at_own_states(orc, width, N, T, M, seed):
    sc = _speed_scene(seed, N, T, M, width)
    g = _plan(sc)
    fh = g["first_hit"]
    n_speed = checked = 0
    for n in range(N):
        want, amb = _discard_at_own_states(orc, sc, g, n)
        if amb:
            continue
        checked += 1
        assert fh[n] == want, (n, fh[n], want)
        if want > 0 and not orc.collide(sc["preset"], *g["sample_traj"][want, n][:3].astype(np.float64),
                                        P.oracle_inputs(sc)[4], tau=want * sc["preset"]["Ts"])[0]:
            n_speed += 1
    assert checked > 0.95 * N and n_speed > 0.1 * N
    assert np.all(np.isinf(g["costs"][fh >= 0])) and np.all(np.isfinite(g["costs"][fh < 0]))
    assert (fh < 0).sum() > 0
    # every step before the discard replays through the oracle
    rs = P.replay_stats(sc, g, np.arange(min(N, 120)))
    assert not rs["bad"], rs["bad"][:5]
    # the winner is the best kept sample
    assert g["status"] == 0 and g["costs"][g["best_idx"]] == np.min(g["costs"])
    # free-running oracle rollouts with the same limits
    o = P.oracle_samples(sc, np.arange(N), record=False)
    assert np.mean(o["first_hit"] == fh) >= 0.95


def test_speed_limits_all_checks_identical():
    """Brute-force variants 0-4, the binned check and the fused check give
    the same discard steps, costs and winner."""
    sc = _speed_scene(84, 2000, 30, 600, 32, box=60.0)
    ref = _plan(sc, 2, record=False)
    assert 0 < np.count_nonzero(ref["first_hit"] < 0) < sc["N"]
    for v, fuse in ((0, 0), (1, 0), (3, 0), (4, 0), (5, 0), (5, 1)):
        r = _plan(sc, v, fuse, record=False)
        np.testing.assert_array_equal(r["first_hit"], ref["first_hit"])
        np.testing.assert_array_equal(r["costs"].view(np.int32), ref["costs"].view(np.int32))
        assert (r["best_idx"], r["status"]) == (ref["best_idx"], ref["status"])
        np.testing.assert_array_equal(r["trajectory"], ref["trajectory"])
        np.testing.assert_array_equal(r["controls"], ref["controls"])


def test_speed_limits_none_kept_is_infeasible():
    """Limits no state after the first step can meet: every sample is
    discarded at h = 1; INFEASIBLE, the lowest index, and the winner's rows
    after h = 1 repeat that state with zero controls."""
    sc = _with(inputs.tiny_scene(85, N=500, T=15, M=30, width=16), v_limits=1, v_min=50.0, v_max=60.0)
    for v, fuse in ((2, 0), (5, 0), (5, 1)):
        r = _plan(sc, v, fuse, record=False)
        assert np.all(r["first_hit"] == 1)
        assert r["status"] == 2 and r["best_idx"] == 0
        np.testing.assert_array_equal(r["trajectory"][2:], np.tile(r["trajectory"][1], (14, 1)))
        assert np.all(r["controls"][1:] == 0)


def test_speed_limits_batch_and_noalloc_match_plan_step():
    import torch
    from paper_1904_06680_gb300 import npp
    scs = [_speed_scene(90 + i, N, T, M, w) for i, (w, N, T, M) in
           enumerate([(16, 700, 20, 150), (32, 333, 33, 40), (64, 129, 12, 301), (32, 96, 8, 0)])]
    p = scs[0]["preset"]
    for sc in scs[1:]:                                   # one handle: one set of limits
        sc["preset"] = dict(sc["preset"], v_min=p["v_min"], v_max=p["v_max"])
    obs_all = np.concatenate([sc["obs"] for sc in scs if sc["obs"].shape[0]])
    offs = np.cumsum([0] + [sc["obs"].shape[0] for sc in scs])
    descs = [dict(state=sc["state"], goal=sc["goal"], N=sc["N"], T=sc["T"], M=sc["obs"].shape[0],
                  width=sc["preset"]["widths"][1], obs_offset=int(offs[i]), seed=sc["seed"],
                  t_index=sc["t_index"]) for i, sc in enumerate(scs)]
    pl = npp.Planner(p, max_N=1, max_T=1, max_M=1)
    B = npp.npp_batch_create(pl.h, npp.make_scenes(descs))
    S = len(descs)
    off = npp.npp_batch_offsets(B, S)
    best = torch.zeros(S * 8, dtype=torch.int32, device="cuda")
    params = torch.zeros(int(off[S, 0]), dtype=torch.float32, device="cuda")
    ctrl = torch.zeros(int(off[S, 1]) * 2, dtype=torch.float32, device="cuda")
    traj = torch.zeros(int(off[S, 2]) * 4, dtype=torch.float32, device="cuda")
    costs = torch.zeros(int(off[S, 3]), dtype=torch.float32, device="cuda")
    fh = torch.zeros(int(off[S, 3]), dtype=torch.int32, device="cuda")
    out = npp.npp_batch_outputs()
    out.best, out.params, out.controls = best.data_ptr(), params.data_ptr(), ctrl.data_ptr()
    out.trajectory, out.costs, out.first_hit = traj.data_ptr(), costs.data_ptr(), fh.data_ptr()
    npp.npp_plan_batch(B, torch.tensor(obs_all, dtype=torch.float32, device="cuda"), out)
    torch.cuda.synchronize()
    bh = best.cpu().view(S, 8)
    n_discard = 0
    for i, (sc, d) in enumerate(zip(scs, descs)):
        r = _plan(sc, record=False)
        a, b = int(off[i, 3]), int(off[i, 3]) + d["N"]
        np.testing.assert_array_equal(fh[a:b].cpu().numpy(), r["first_hit"])
        np.testing.assert_array_equal(costs[a:b].cpu().numpy(), r["costs"])
        assert int(bh[i, 0]) == r["best_idx"] and int(bh[i, 1]) == r["status"]
        n_discard += int(np.count_nonzero(r["first_hit"] >= 0))
        # the allocation-free entry point
        N, T, M = d["N"], d["T"], d["M"]
        cfg = npp.make_config(sc["preset"], N, T, max(M, 1))
        nb = torch.zeros(8, dtype=torch.int32, device="cuda")
        ncost = torch.zeros(N, dtype=torch.float32, device="cuda")
        nfh = torch.zeros(N, dtype=torch.int32, device="cuda")
        o = npp.npp_outputs()
        o.best, o.costs, o.first_hit = nb.data_ptr(), ncost.data_ptr(), nfh.data_ptr()
        obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda") if M else None
        npp.npp_plan_step_noalloc(cfg, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], sc["t_index"], None, o)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(nfh.cpu().numpy(), r["first_hit"])
        assert int(nb[0]) == r["best_idx"]
    assert n_discard > 0
    npp.npp_batch_destroy(B)
    pl.close()


def test_invalid_variant_fields():
    from paper_1904_06680_gb300 import npp
    p = inputs.planner(16)
    for bad in (dict(feature_frame=2), dict(v_limits=3), dict(v_limits=1, v_min=2.0, v_max=1.0),
                dict(v_limits=1, v_min=float("nan"), v_max=1.0)):
        with pytest.raises(npp.NppError):
            npp.Planner(dict(p, **bad), max_N=8, max_T=4, max_M=1)


def test_closed_loop_respects_speed_limit():
    """Obstacle-free run towards a goal 60 m ahead with v_max = 3 m/s: the
    winner's speeds stay within the limit (plant in FP64: 1e-3 slack)."""
    import torch
    from paper_1904_06680_gb300 import npp
    p = dict(inputs.planner(16), v_limits=1, v_min=-1.0, v_max=3.0)
    N, T = 4096, 30
    pl = npp.Planner(p, max_N=N, max_T=T, max_M=1)
    obs = torch.zeros(1, 4, dtype=torch.float32, device="cuda")
    obs[0, :2] = 1e4
    start = [0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    goal = [60.0, 0.0, 0.0, 0.0]
    L = npp.npp_loop_create(pl.h, start, [goal], inputs.EPS, obs, 1, N, T, 91)
    npp.npp_loop_run(L, 80)
    log = npp.npp_loop_log(L)
    st = npp.npp_loop_read(L)
    npp.npp_loop_destroy(L)
    pl.close()
    assert st["n_infeasible"] == 0
    assert np.max(log[:, 3]) <= 3.0 + 1e-3 and np.min(log[:, 3]) >= -1.0 - 1e-3
    assert np.max(log[:, 3]) > 2.5                  # it does drive near the limit
    assert log[-1, 0] > 10.0
