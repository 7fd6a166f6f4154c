"""Helpers for the GPU-vs-oracle parity tests (not a test module).

Tolerances (from the arithmetic; the paper fixes no precision):
  * sampled parameters: bit-exact (integer Philox + the FP32 sampler spec);
  * one replayed step -- the oracle (FP64) takes the GPU's own FP32 state and
    previous controls at step h: the controls it computes within 2e-5
    absolute of the GPU's (an FP32 dot product of up to 64 terms of size O(1)
    plus tanh carries a few 1e-7), and its Euler step from that state with
    the GPU's applied controls within 2e-6 relative (floors of 1 m, 1 rad,
    1 m/s: one FP32 update of values up to ~50 m) plus Ts |v| 3e-6 absolute
    (the step's sin/cos of the heading and tan of the steering carry at most
    1e-6 and 2e-6, tests/test_gpu_math.py); the two checks are separate so
    that an allowed control difference is not counted again in the state;
    steps where the heading error feature sits within 1e-4 rad of its +-pi
    wrap are ambiguous (FP32 and FP64 may wrap to opposite sides);
  * free-running trajectories: within 1e-4 relative, same floors, wherever
    the oracle's own FP64 trajectory is stable.  A rollout whose controls
    feed back through a random network can amplify a rounding-sized change
    of its inputs a million-fold over 100 steps (chaotic samples); no FP32
    computation tracks such a sample to 1e-4, and CUDA's correctly rounded
    tanhf/tanf/sincosf in place of the SFU forms change nothing measurable
    (fractions within 1e-4 at N=16384, T=40: 95.4 % vs 94.1 %; N=65536,
    T=100: 82.7 % vs 82.8 %).  So each sample's sensitivity kappa is probed
    in the oracle itself (largest relative change of its FP64 trajectory
    under four input changes of relative size 1e-6: goal position, start
    speed and last controls, two random sign patterns on the parameters),
    and the GPU trajectory must lie within max(1e-4, 10 kappa) of the
    oracle's -- it is the exact result of a problem perturbed by about
    1e-5 (backward stable).  A first collision step may differ only for a
    sample with kappa >= 1e-3.  Required of the winner and of >= 99 % of the
    compared samples (the probes sample a few of the directions rounding
    takes);
  * collision flags: the oracle re-evaluates the GPU's states; a decision is
    ambiguous only when some point lies within 1e-4 m of a face;
  * cost: every collision-free sample's GPU cost within 1e-5 relative of
    the oracle's cost formula evaluated at the GPU's own final state and
    controls; the GPU's best cost no worse than (1 + 1e-5) x the oracle's
    best over the samples where GPU and oracle agree.
"""
import math

import numpy as np

FLOORS = np.array([1.0, 1.0, 1.0, 1.0])
REPLAY_CTRL_ATOL = 2e-5
REPLAY_RTOL = 2e-6
FUNC_ERR = 3e-6          # sin/cos (1e-6) and tan (2e-6) bounds of the step's FP32 functions
TRAJ_RTOL = 1e-4
FACE_MARGIN = 1e-4
WRAP_MARGIN = 1e-4
COST_RTOL = 1e-5
COND_EPS = 1e-6          # relative size of the oracle's input probes
COND_FACTOR = 10.0       # GPU error allowed per unit of the oracle's own sensitivity
COND_FH = 1e-3           # sensitivity from which the first collision step may differ
CONSISTENT_FRAC = 0.99


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
            a_o, _ = orc.step(p, th, z, ap, goal_ev, h, T)
            zn_o = orc.euler_step(p, z, a_g)
            ec = float(np.max(np.abs(a_o - a_g)))
            es = float(np.max(np.abs(zn_g - zn_o) / (np.maximum(np.abs(zn_o), FLOORS) * REPLAY_RTOL
                                                       + p["Ts"] * abs(z[3]) * FUNC_ERR))) * REPLAY_RTOL
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


def conditioning(sc, idx, o, eps=COND_EPS):
    """How far the oracle's own FP64 trajectory of each sample moves when its
    inputs move by eps: the goal position scaled by (1 + eps); the start
    speed raised by eps m/s with the last controls moved by -+eps; the
    parameters scaled by (1 -+ eps) in two fixed random sign patterns.
    Returns per sample the largest relative change of any state up to its
    first collision over the four probes (floors as above), inf when the
    first collision step changes.  `o` holds the unperturbed rollouts of
    idx (warm starts are not probed: idx must be sampled parameters)."""
    from oracle import oracle as orc
    st, gl, ob, goal_ev, obs_ev = oracle_inputs(sc)
    T = sc["T"]
    p = sc["preset"]
    kappa = np.zeros(len(idx))
    g1 = goal_ev.copy()
    g1[:2] *= (1.0 + eps)
    ap1 = np.clip(st[4:6] + np.array([-eps, eps]), -1.0, 1.0)
    z0 = [0, 0, 0, st[3]]
    runs = [orc.rollout_samples(p, sc["seed"], sc["t_index"], np.asarray(idx, np.int32), z0, st[4:6], g1,
                                obs_ev, T, record=True),
            orc.rollout_samples(p, sc["seed"], sc["t_index"], np.asarray(idx, np.int32), [0, 0, 0, st[3] + eps],
                                ap1, goal_ev, obs_ev, T, record=True)]
    nt = orc.n_theta(p)
    th = np.stack([orc.theta(sc["seed"], sc["t_index"], int(n), nt).astype(np.float64) for n in idx])
    for pat in (1, 2):
        sign = np.random.default_rng(pat).choice([-1.0, 1.0], th.shape)
        runs.append(orc.rollout_theta(p, th * (1.0 + eps * sign), z0, st[4:6], goal_ev, obs_ev, T))
    for q in runs:
        for k in range(len(idx)):
            if int(q["first_hit"][k]) != int(o["first_hit"][k]):
                kappa[k] = np.inf
                continue
            fh = int(o["first_hit"][k])
            last = T if fh < 0 else fh
            kappa[k] = max(kappa[k], float(np.max(_rel(q["traj"][k][: last + 1], o["traj"][k][: last + 1]))))
    return kappa


def traj_errors(sc, g, o, idx):
    """Largest relative difference (floors as above) between the GPU's and
    the oracle's free-running trajectory of each sample, up to the first
    collision; inf where the first collision steps differ."""
    T = sc["T"]
    err = np.full(len(idx), np.inf)
    for k, n in enumerate(idx):
        fh_g, fh_o = int(g["first_hit"][n]), int(o["first_hit"][k])
        if fh_g != fh_o:
            continue
        last = T if fh_g < 0 else fh_g
        err[k] = float(np.max(_rel(g["sample_traj"][: last + 1, n].astype(np.float64), o["traj"][k][: last + 1])))
    return err


def consistent(err, kappa):
    """Per sample: the GPU trajectory lies within max(1e-4, 10 kappa) of the
    oracle's, or the first collision steps differ on a sample with kappa >=
    1e-3."""
    with np.errstate(invalid="ignore"):
        close = err <= np.maximum(TRAJ_RTOL, COND_FACTOR * kappa)
    return close | (~np.isfinite(err) & (kappa >= COND_FH))


def traj_check(sc, g, idx, o=None):
    """The free-running trajectory rule on samples idx (winner included by
    the caller): returns (consistent fraction, per-sample consistency,
    errors, kappa, oracle rollouts)."""
    if o is None:
        o = oracle_samples(sc, idx)
    err = traj_errors(sc, g, o, idx)
    kap = conditioning(sc, idx, o)
    ok = consistent(err, kap)
    return float(ok.mean()), ok, err, kap, o


def cost_at_gpu_states(sc, g, idx):
    """Relative difference between each collision-free sample's GPU cost and
    the oracle's cost formula evaluated (FP64) at the GPU's own final state
    and applied controls; nan for collided samples."""
    from oracle import oracle as orc
    _, _, _, goal_ev, _ = oracle_inputs(sc)
    T = sc["T"]
    out = np.full(len(idx), np.nan)
    for k, n in enumerate(idx):
        if int(g["first_hit"][n]) >= 0:
            continue
        c_o = orc.cost(sc["preset"], g["sample_traj"][T, n].astype(np.float64),
                       g["sample_ctrl"][:T, n].astype(np.float64), goal_ev)
        out[k] = abs(float(g["costs"][n]) - c_o) / max(1.0, abs(c_o))
    return out


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
               gpu_pick_in_agree=bool(agree_cost[b]), gpu_best_cost=float(g["best_cost"]),
               ok=bool(float(g["best_cost"]) <= best_u * (1 + COST_RTOL) + COST_RTOL))
    return res
