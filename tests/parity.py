"""Helpers for the GPU-vs-oracle parity tests (not a test module).

Tolerances (from the arithmetic; the paper fixes no precision):
  * sampled parameters: bit-exact (integer Philox + the FP32 sampler spec);
  * one replayed step -- the oracle (FP64) takes the GPU's own FP32 state and
    previous controls at step h and computes the controls and the state at
    h+1: controls within 2e-5 absolute (an FP32 dot product of up to 64 terms
    of size O(1) plus tanh carries a few 1e-7), state within 2e-6 relative
    with floors of 1 m, 1 rad, 1 m/s (one FP32 Euler update of values up to
    ~50 m); steps where the heading error feature sits within 1e-4 rad of its
    +-pi wrap are ambiguous (FP32 and FP64 may wrap to opposite sides);
  * free-running trajectories: within 1e-4 relative, same floors;
  * collision flags: the oracle re-evaluates the GPU's states; a decision is
    ambiguous only when some point lies within 1e-4 m of a face;
  * cost of the chosen sample: within 1e-5 relative of the oracle's best
    over the samples where GPU and oracle agree.
"""
import math

import numpy as np

FLOORS = np.array([1.0, 1.0, 1.0, 1.0])
REPLAY_CTRL_ATOL = 2e-5
REPLAY_RTOL = 2e-6
TRAJ_RTOL = 1e-4
FACE_MARGIN = 1e-4
WRAP_MARGIN = 1e-4
COST_RTOL = 1e-5


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gpu_plan(sc, record=True, warm=None, device=0):
    import torch
    from paper_1904_06680_gb300 import npp
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    dev = torch.device("cuda", device)
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=max(M, 1), device=device,
                     record_samples=record)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device=dev) if M else None
    w = None if warm is None else torch.tensor(warm, dtype=torch.float32, device=dev)
    pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"], warm=w)
    torch.cuda.synchronize()
    r = pl.result(N, T)
    pl.close()
    return r


def oracle_inputs(sc):
    from oracle import oracle as orc
    st, gl, ob = f32(sc["state"]), f32(sc["goal"]), f32(sc["obs"]).reshape(-1, 4)
    goal_ev, obs_ev = orc.frame_to_ev(st, gl, ob)
    return st, gl, ob, goal_ev, obs_ev


def oracle_samples(sc, idx, warm=None, record=True):
    from oracle import oracle as orc
    st, gl, ob, goal_ev, obs_ev = oracle_inputs(sc)
    return orc.rollout_samples(sc["preset"], sc["seed"], sc["t_index"], np.asarray(idx, np.int32),
                               [0, 0, 0, st[3]], st[4:6], goal_ev, obs_ev, sc["T"],
                               warm=None if warm is None else f32(warm), record=record)


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), FLOORS)


def replay_stats(sc, g, idx):
    """Per-step replay of the GPU's own states through the oracle."""
    from oracle import oracle as orc
    p = sc["preset"]
    T = sc["T"]
    st, gl, ob, goal_ev, obs_ev = oracle_inputs(sc)
    nt = orc.n_theta(p)
    worst_ctrl = 0.0
    worst_state = 0.0
    n_steps = n_amb = 0
    bad = []
    for n in idx:
        th = orc.theta(sc["seed"], sc["t_index"], int(n), nt).astype(np.float64)
        fh = int(g["first_hit"][n])
        last = T if fh < 0 else fh          # control steps taken: 0 .. last-1
        ap = st[4:6].copy()
        for h in range(last):
            z = g["sample_traj"][h, n].astype(np.float64)
            a_g = g["sample_ctrl"][h, n].astype(np.float64)
            zn_g = g["sample_traj"][h + 1, n].astype(np.float64)
            dphi = goal_ev[2] - z[2]
            if abs(math.remainder(dphi - math.pi, 2 * math.pi)) < WRAP_MARGIN:
                n_amb += 1
                ap = a_g
                continue
            a_o, zn_o = orc.step(p, th, z, ap, goal_ev, h, T)
            ec = float(np.max(np.abs(a_o - a_g)))
            es = float(np.max(_rel(zn_g, zn_o)))
            worst_ctrl = max(worst_ctrl, ec)
            worst_state = max(worst_state, es)
            if ec > REPLAY_CTRL_ATOL or es > REPLAY_RTOL:
                bad.append((int(n), h, ec, es))
            n_steps += 1
            ap = a_g
    return dict(worst_ctrl=worst_ctrl, worst_state=worst_state, steps=n_steps, ambiguous=n_amb,
                bad=bad)


def flag_stats(sc, g, idx):
    """Collision decisions at the GPU's own states, re-evaluated in FP64."""
    from oracle import oracle as orc
    p = sc["preset"]
    T = sc["T"]
    _, _, _, _, obs_ev = oracle_inputs(sc)
    checked = amb = 0
    bad = []
    for n in idx:
        fh = int(g["first_hit"][n])
        last = T if fh < 0 else fh
        for h in range(last + 1):
            z = g["sample_traj"][h, n].astype(np.float64)
            flag, n_clear, n_near = orc.collide(p, z[0], z[1], z[2], obs_ev, tau=h * p["Ts"],
                                                margin=FACE_MARGIN)
            want = (h == fh)
            if n_clear == 0 and n_near > 0:
                amb += 1
                continue
            checked += 1
            if flag != want:
                bad.append((int(n), h, flag, want))
    return dict(checked=checked, ambiguous=amb, bad=bad)


def traj_stats(sc, g, o, idx):
    """Free-running comparison of sample trajectories, controls and costs."""
    T = sc["T"]
    ok = []
    for k, n in enumerate(idx):
        fh_g, fh_o = int(g["first_hit"][n]), int(o["first_hit"][k])
        if fh_g != fh_o:
            ok.append(False)
            continue
        last = T if fh_g < 0 else fh_g
        zg = g["sample_traj"][: last + 1, n].astype(np.float64)
        zo = o["traj"][k][: last + 1]
        good = bool(np.all(_rel(zg, zo) <= TRAJ_RTOL))
        if fh_g < 0:
            good = good and abs(g["costs"][n] - o["cost"][k]) <= TRAJ_RTOL * max(1.0, abs(o["cost"][k]))
        ok.append(good)
    return np.array(ok)


def winner_check(g, o_cost, o_fh):
    """GPU's pick vs the oracle's best over samples where both agree."""
    gc = g["costs"].astype(np.float64)
    gfh = g["first_hit"]
    agree = (gfh == o_fh)
    free = agree & (gfh < 0)
    with np.errstate(invalid="ignore"):
        diff = np.where(free, np.abs(gc - o_cost), np.inf)
    agree_cost = free & (diff <= COST_RTOL * np.maximum(1.0, np.abs(o_cost)))
    res = dict(agree_frac=float(agree.mean()), n_free=int((gfh < 0).sum()))
    if not np.any(o_fh < 0):
        res["infeasible"] = True
        return res
    best_u = np.min(np.where(agree_cost, o_cost, np.inf))
    b = g["best_idx"]
    res.update(best_unambiguous=float(best_u), gpu_pick=int(b), gpu_pick_oracle_cost=float(o_cost[b]),
               gpu_pick_in_agree=bool(agree_cost[b]))
    return res
