"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Small instances are compared on every sample (several blocks and a ragged
tail); the full-size workloads on every sample too where the oracle is fast
enough, otherwise on sampled indices.  Tolerances are documented in
tests/parity.py.
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
    from paper_1904_06680_gb300 import npp
    npp.lib()


# ------------------------------------------------------------------ sampler
@pytest.mark.parametrize("nt", [450, 1410, 4866, 7])
def test_sampled_parameters_bit_exact(orc, nt):
    import torch
    from paper_1904_06680_gb300 import npp
    rng = np.random.default_rng(nt)
    for _ in range(3):
        seed = int(rng.integers(0, 2 ** 63))
        t = int(rng.integers(0, 2 ** 32))
        stream = int(rng.integers(0, 4))
        n0 = int(rng.integers(0, 2 ** 31 - 100))
        K = 37
        out = torch.empty(K * nt, dtype=torch.float32, device="cuda")
        npp.npp_sample_params(seed, t, stream, n0, K, nt, out)
        g = out.view(K, nt).cpu().numpy()
        for k in range(K):
            ref = orc.theta(seed, t, n0 + k, nt, stream=stream)
            assert np.array_equal(g[k].view(np.uint32), ref.view(np.uint32)), (seed, t, n0 + k)


def test_sampled_parameters_bulk(orc):
    """65536 x 450 draws: bit-exact on a strided subset, moments on all."""
    import torch
    from paper_1904_06680_gb300 import npp
    K, nt = 65536, 450
    out = torch.empty(K * nt, dtype=torch.float32, device="cuda")
    npp.npp_sample_params(0x5EED0000, 3, 0, 0, K, nt, out)
    g = out.view(K, nt)
    for k in range(0, K, 4099):
        assert np.array_equal(g[k].cpu().numpy(), orc.theta(0x5EED0000, 3, k, nt))
    x = g.double()
    assert abs(x.mean().item()) < 5 / math.sqrt(K * nt)
    assert abs(x.var().item() - 1) < 5 * math.sqrt(2 / (K * nt))


# ------------------------------------------------------------------ small plans
SMALL = [(16, 300, 20, 40, 11), (32, 150, 24, 60, 12), (64, 70, 18, 33, 13), (16, 1, 5, 7, 14),
         (32, 33, 1, 0, 15)]


@pytest.mark.parametrize("width,N,T,M,seed", SMALL)
def test_plan_parity_small(orc, width, N, T, M, seed):
    sc = inputs.tiny_scene(seed, N=N, T=T, M=M, width=width)
    g = P.gpu_plan(sc)
    idx = np.arange(N)
    o = P.oracle_samples(sc, idx)
    # winner parameters and summary record
    nt = orc.n_theta(sc["preset"])
    assert np.array_equal(g["params"], orc.theta(sc["seed"], sc["t_index"], g["best_idx"], nt))
    assert g["costs"][g["best_idx"]] == np.min(g["costs"]) or g["status"] == 2
    # per-step replay of every step of every sample
    rs = P.replay_stats(sc, g, idx)
    assert not rs["bad"], rs["bad"][:5]
    # collision decisions at the GPU's states
    fs = P.flag_stats(sc, g, idx)
    assert not fs["bad"], fs["bad"][:5]
    # free-running trajectories against the oracle's own sensitivity, the
    # winner's included
    frac, ok, err, kap, _ = P.traj_check(sc, g, idx, o)
    assert frac >= P.CONSISTENT_FRAC, (frac, err[~ok][:5], kap[~ok][:5])
    assert ok[g["best_idx"]], (err[g["best_idx"]], kap[g["best_idx"]])
    # costs at the GPU's own states; the chosen sample
    ca = P.cost_at_gpu_states(sc, g, idx)
    assert np.nanmax(ca, initial=0.0) <= P.COST_RTOL, np.nanmax(ca)
    wc = P.winner_check(g, o["cost"], o["first_hit"])
    if not wc.get("infeasible"):
        assert wc["ok"], wc
    # winner trajectory and controls in the world frame
    b = g["best_idx"]
    fh = int(g["first_hit"][b])
    last = T if fh < 0 else fh
    c, s = math.cos(np.float32(sc["state"][2])), math.sin(np.float32(sc["state"][2]))
    ev = g["sample_traj"][:, b].astype(np.float64)
    x0, y0 = np.float32(sc["state"][0]), np.float32(sc["state"][1])
    for h in range(T + 1):
        z = ev[min(h, last)]
        w = [x0 + c * z[0] - s * z[1], y0 + s * z[0] + c * z[1]]
        assert np.allclose(g["trajectory"][h, :2], w, rtol=1e-6, atol=1e-4)
    assert np.array_equal(g["controls"][:last], g["sample_ctrl"][:last, b])
    assert np.all(g["controls"][last:] == 0)


def test_plan_warm_start(orc):
    sc = inputs.tiny_scene(21, N=100, T=15, M=30, width=32)
    nt = orc.n_theta(sc["preset"])
    warm = np.zeros(nt, np.float32)
    warm[-2:] = [0.0, math.atanh(0.2)]
    g = P.gpu_plan(sc, warm=warm)
    o = P.oracle_samples(sc, [0], warm=warm)
    assert int(g["first_hit"][0]) == int(o["first_hit"][0])
    if o["first_hit"][0] < 0:
        assert abs(g["costs"][0] - o["cost"][0]) <= 1e-4 * max(1, abs(o["cost"][0]))
    if g["best_idx"] == 0:
        assert np.array_equal(g["params"], warm)


def test_plan_infeasible(orc):
    """Every sample collides: INFEASIBLE and the longest survivor."""
    sc = inputs.tiny_scene(22, N=96, T=30, M=0, width=16)
    rng = np.random.default_rng(22)
    ang = rng.uniform(-math.pi, math.pi, 3000)
    rad = rng.uniform(3.5, 6.0, 3000)
    st = sc["state"]
    obs = np.zeros((3000, 4))
    obs[:, 0] = st[0] + rad * np.cos(ang)
    obs[:, 1] = st[1] + rad * np.sin(ang)
    obs[:, 2] = -2.0 * np.cos(ang)
    obs[:, 3] = -2.0 * np.sin(ang)
    sc["obs"] = obs
    g = P.gpu_plan(sc)
    o = P.oracle_samples(sc, np.arange(96))
    assert np.all(g["first_hit"] >= 0) and g["status"] == 2
    assert g["best_idx"] == int(np.argmax(g["first_hit"]))
    assert np.isinf(g["best_cost"])
    assert np.mean(g["first_hit"] == o["first_hit"]) > 0.9
    fh = int(g["first_hit"][g["best_idx"]])
    assert np.all(g["controls"][fh:] == 0)
    # a point inside the car at h = 0
    sc["obs"] = np.array([[st[0], st[1], 0.0, 0.0]])
    g2 = P.gpu_plan(sc)
    assert g2["status"] == 2 and np.all(g2["first_hit"] == 0) and g2["best_idx"] == 0


def test_invalid_arguments():
    import torch
    from paper_1904_06680_gb300 import inputs as I, npp
    p = I.planner(16)
    with pytest.raises(npp.NppError):
        npp.Planner(dict(p, widths=(8, 24, 24, 2)), 10, 10, 10)
    pl = npp.Planner(p, max_N=64, max_T=10, max_M=8)
    obs = torch.zeros(8, 4, device="cuda")
    for bad in [dict(N=0), dict(N=65), dict(T=0), dict(T=11)]:
        kw = dict(N=10, T=5)
        kw.update(bad)
        with pytest.raises(npp.NppError) as ei:
            pl.plan([0, 0, 0, 0, 0, 0], [5, 0, 0, 0], obs, kw["N"], kw["T"], 1)
        assert ei.value.status == npp.NPP_INVALID_ARG
    with pytest.raises(npp.NppError):
        pl.plan([0, 0, float("nan"), 0, 0, 0], [5, 0, 0, 0], obs, 10, 5, 1)
    with pytest.raises(npp.NppError):
        pl.plan([0, 0, 0, 0, 2.0, 0], [5, 0, 0, 0], obs, 10, 5, 1)
    pl.close()


# ------------------------------------------------------------------ full sizes
def test_single_scene_full(orc):
    """The 1-scene workload (N=256, T=20, 8-16-16-2, M=200): every sample."""
    sc = inputs.scene_single(0)
    g = P.gpu_plan(sc)
    idx = np.arange(sc["N"])
    o = P.oracle_samples(sc, idx)
    rs = P.replay_stats(sc, g, idx)
    assert not rs["bad"], rs["bad"][:5]
    fs = P.flag_stats(sc, g, idx)
    assert not fs["bad"], fs["bad"][:5]
    frac, ok, err, kap, _ = P.traj_check(sc, g, idx, o)
    assert frac >= P.CONSISTENT_FRAC, (frac, err[~ok][:5], kap[~ok][:5])
    assert ok[g["best_idx"]]
    ca = P.cost_at_gpu_states(sc, g, idx)
    assert np.nanmax(ca, initial=0.0) <= P.COST_RTOL, np.nanmax(ca)
    wc = P.winner_check(g, o["cost"], o["first_hit"])
    assert wc["ok"], wc


def _full_size(sc, fh_agree_min):
    """Every sample's collision status and cost from the oracle; per-step
    replay, flags at the GPU's states, the trajectory rule and the cost at
    the GPU's states on 1024 sampled indices plus the winner."""
    g = P.gpu_plan(sc)
    N = sc["N"]
    o = P.oracle_samples(sc, np.arange(N), record=False)
    wc = P.winner_check(g, o["cost"], o["first_hit"])
    assert wc["agree_frac"] >= fh_agree_min, wc
    assert wc["ok"], wc
    idx = np.random.default_rng(0).choice(N, 1024, replace=False)
    idx = np.union1d(idx, [g["best_idx"]])
    kb = int(np.searchsorted(idx, g["best_idx"]))
    rs = P.replay_stats(sc, g, idx)
    assert not rs["bad"], rs["bad"][:5]
    fs = P.flag_stats(sc, g, idx)
    assert not fs["bad"], fs["bad"][:5]
    frac, ok, err, kap, o2 = P.traj_check(sc, g, idx)
    assert frac >= P.CONSISTENT_FRAC, (frac, err[~ok][:5], kap[~ok][:5])
    assert ok[kb], (err[kb], kap[kb])
    # where GPU and oracle disagree on the first collision, the oracle's own
    # first collision moves under the 1e-6 probes as well
    assert np.all(kap[o2["first_hit"] != g["first_hit"][idx]] >= P.COND_FH)
    ca = P.cost_at_gpu_states(sc, g, idx)
    assert np.nanmax(ca, initial=0.0) <= P.COST_RTOL, np.nanmax(ca)
    return g


def test_course_full_size(orc):
    """The closed-loop course workload at full size (N=16384, T=40,
    8-32-32-2, M=2000), as the benchmark launches it (binned collision
    check)."""
    _full_size(inputs.scene_course(0), 0.99)


def test_large_full_size(orc):
    """The largest workload at full size (N=65536, T=100, 8-64-64-2, M=8192
    over 80 x 80 m, 20 % moving), as the benchmark launches it (binned
    collision check).  Over T=100 steps more samples are sensitive: the
    first collision step agrees on >= 98 % of all samples, and on the
    sampled indices every disagreement is on a sample whose own oracle
    trajectory changes its first collision under the 1e-6 probes."""
    _full_size(inputs.scene_large(0), 0.98)


def test_paper_horizon(orc):
    """The paper's horizon H = 200 with its vehicle (Experiment 3's road:
    16 bounds and a car ahead at 20 km/h; 8-16-16-2, N = 4096): every
    sample's status and cost from the oracle; per-step replay, decisions at
    the GPU's states, the trajectory rule and the cost at the GPU's states
    on 1024 sampled indices and the winner."""
    _full_size(inputs.scene_paper_road(True, N=4096), 0.95)


def test_large_point_set_from_global_memory(orc):
    """More points than shared memory holds: the collision kernel reads an
    L2-resident copy; every sample against the oracle."""
    sc = inputs.tiny_scene(32, N=200, T=15, M=16001, width=16, box=120.0)
    g = P.gpu_plan(sc)
    idx = np.arange(sc["N"])
    o = P.oracle_samples(sc, idx, record=False)
    wc = P.winner_check(g, o["cost"], o["first_hit"])
    assert wc["agree_frac"] >= 0.99, wc
    assert 0 < np.sum(g["first_hit"] >= 0) < sc["N"]
    if not wc.get("infeasible"):
        assert wc["gpu_pick_oracle_cost"] <= wc["best_unambiguous"] * (1 + P.COST_RTOL) + P.COST_RTOL, wc
    fs = P.flag_stats(sc, g, idx[:40])
    assert not fs["bad"], fs["bad"][:5]


def test_collide_variants_identical():
    """The launch variants of the collision and trajectory kernels compute
    the same values."""
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.tiny_scene(31, N=1000, T=25, M=301, width=32, box=30.0)
    N, T = sc["N"], sc["T"]
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=obs.shape[0])
    res = []
    for v, tv in [(0, 0), (1, 1), (2, 0), (0, 1), (1, 0), (3, 0), (4, 0), (5, 0), (5, 1), (2, 2), (3, 3), (4, 4),
                  (5, 4)]:
        npp.npp_set_option(pl.h, "collide_variant", v)
        npp.npp_set_option(pl.h, "traj_variant", tv)
        pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
        torch.cuda.synchronize()
        r = pl.result(N, T)
        res.append((r["costs"].copy(), r["first_hit"].copy(), r["best_idx"], r["trajectory"].copy()))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1]) and r[2] == res[0][2]
        assert np.array_equal(r[3], res[0][3])
    assert 0 < np.sum(res[0][1] >= 0) < N
    with pytest.raises(npp.NppError):
        npp.npp_set_option(pl.h, "collide_variant", 6)
    npp.npp_set_option(pl.h, "collide_variant", -1)
    pl.close()


@pytest.mark.parametrize("width", [64, 32, 16])
def test_trajectory_launch_shapes_identical(width):
    """Every launch shape of the trajectory kernel gives the same bits:
    per-sample states, controls, costs, first collisions and the winner.
    At width 64 the default keeps half of each lane's layer-2 weights in
    shared memory and shape 4 all in registers; at width 32 shape 4 keeps 5
    of each lane's 8 layer-2 input quads in shared memory."""
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.tiny_scene(33, N=700, T=30, M=250, width=width, box=30.0)
    N, T = sc["N"], sc["T"]
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=obs.shape[0], record_samples=True)
    res = []
    for tv in range(5):
        npp.npp_set_option(pl.h, "traj_variant", tv)
        pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
        torch.cuda.synchronize()
        res.append(pl.result(N, T))
    for r in res[1:]:
        for k in ("sample_traj", "sample_ctrl", "costs", "first_hit", "params", "trajectory"):
            assert np.array_equal(r[k], res[0][k]), k
        assert r["best_idx"] == res[0]["best_idx"]
    assert 0 < np.sum(res[0]["first_hit"] >= 0) < N
    with pytest.raises(npp.NppError):
        npp.npp_set_option(pl.h, "traj_variant", 5)
    pl.close()


def test_steering_rate_limit_on_every_rollout():
    """Fig. 8: the applied normalised steering moves by at most
    delta_rate_max Ts / delta_max per step (and stays in [-1, 1]) in every
    step of every sample of a full-size plan step."""
    sc = inputs.scene_course(0)
    g = P.gpu_plan(sc, record=True)
    p = sc["preset"]
    r = np.float32(p["delta_rate_max"] * p["Ts"] / p["delta_max"])
    a0 = g["sample_ctrl"][:, :, 0]                        # [T][N]
    prev = np.vstack([np.full((1, a0.shape[1]), np.float32(sc["state"][4])), a0[:-1]])
    fh = g["first_hit"]
    live = np.arange(sc["T"])[:, None] < np.where(fh < 0, sc["T"], fh)[None, :]
    step = np.abs(a0 - prev)[live]
    assert step.max() <= r * (1 + 2 ** -22) + 2 ** -23, step.max()
    assert np.abs(a0[live]).max() <= 1.0
    assert np.mean(step >= r * (1 - 1e-6)) > 0.1           # the limit binds often
