"""The learned sampling proposal on the GPU against the oracle: the
tensor-core GEMM, the network's forward pass, gradients and Adam update,
the scene encoding, and the mixed plan step (proposal samples bit-exact)."""
import math
import os
import sys

import numpy as np
import pytest

from oracle import proposal as OP
from paper_1904_06680_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
import parity  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 256, 128), (384, 384, 320), (128, 1024, 256),
                                   (1024, 256, 512), (512, 128, 1024), (768, 512, 192), (256, 768, 64),
                                   (640, 1280, 576)])
def test_gemm_bf16_against_fp64(M, N, K):
    """C = A B^T against FP64 within K 2^-22 sum |a b|: 128- and 256-wide
    tiles, one or several row and column tiles, also with fewer K blocks
    than pipeline stages."""
    import torch
    from paper_1904_06680_gb300 import npp
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    npp.npp_gemm_bf16(A.cuda(), B.cuda(), C, M, N, K)
    torch.cuda.synchronize()
    npp.npp_gemm_status()
    ref = A.double() @ B.double().T
    bound = (A.double().abs() @ B.double().abs().T) * (K * 2.0 ** -22) + 1e-30
    err = (C.cpu().double() - ref).abs()
    assert torch.all(err <= bound), float((err / bound).max())


def test_gemm_rejects_bad_shapes():
    import torch
    from paper_1904_06680_gb300 import npp
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 128, device="cuda")
    for M, N, K in [(100, 128, 64), (128, 100, 64), (128, 128, 48)]:
        with pytest.raises(npp.NppError):
            npp.npp_gemm_bf16(A, A, C, M, N, K)


def _rand_problem(B, seed):
    rng = np.random.default_rng(seed)
    params = OP.init_params(seed, out_scale=0.5)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.standard_normal(params[k].shape) * 0.2
    X = np.concatenate([rng.uniform(0, 1, (B, 64)), rng.standard_normal((B, 8))], axis=1)
    theta = rng.standard_normal((B, OP.N_THETA)) * 1.3
    vec = OP.pack(params).astype(np.float32)
    return OP.unpack(vec.astype(np.float64)), vec, X.astype(np.float32), theta.astype(np.float32)


def _net(B):
    from paper_1904_06680_gb300 import proposal
    return proposal.ProposalNet(batch=B, ls_min=OP.LS_MIN, ls_max=OP.LS_MAX)


def test_forward_against_oracle():
    import torch
    B = 256
    params, vec, X, _ = _rand_problem(B, 1)
    net = _net(B)
    net.set_params(vec)
    for n in (B, 77):
        mean, std = net.forward(torch.tensor(X[:n], device="cuda"))
        mu_o, sd_o = OP.mean_std(params, X[:n].astype(np.float64))
        c = OP.forward(params, X[:n].astype(np.float64))
        scale = np.max(np.abs(c["Y"]))
        assert np.max(np.abs(mean.cpu().numpy() - mu_o)) <= 1e-2 * scale
        assert np.max(np.abs(np.log(std.cpu().numpy()) - np.log(sd_o))) <= 1e-2 * scale
    net.close()


@pytest.mark.parametrize("B", [256, 4096])
def test_gradients_and_loss_against_oracle(B):
    """Loss and every gradient against the FP64 oracle; the weight gradients
    come from GEMMs with K (the batch) split into 2 (B = 256) or 16-32
    slices (B = 4096) summed in slice order, so a repeated step gives the
    same gradient bits."""
    import torch
    params, vec, X, theta = _rand_problem(B, 2)
    net = _net(B)
    net.set_params(vec)
    xd, td = torch.tensor(X, device="cuda"), torch.tensor(theta, device="cuda")
    loss = net.train_step(xd, td, 0.0)
    g_gpu = OP.unpack(net.grads().astype(np.float64))
    net.train_step(xd, td, 0.0)
    assert np.array_equal(OP.pack(OP.unpack(net.grads().astype(np.float64))), OP.pack(g_gpu))
    c = OP.forward(params, X.astype(np.float64))
    want = OP.nll(c, theta)
    assert abs(float(loss.item()) - want) <= 1e-4 * abs(want) + 1e-5
    g_o = OP.backward(params, c, theta)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        rel = np.linalg.norm(g_gpu[k] - g_o[k]) / max(np.linalg.norm(g_o[k]), 1e-30)
        assert rel <= 2e-2, (k, rel)
    # lr = 0 leaves the parameters unchanged
    np.testing.assert_array_equal(net.params(), vec)
    net.close()


def test_adam_updates_against_oracle():
    import torch
    B = 128
    params, vec, X, theta = _rand_problem(B, 3)
    net = _net(B)
    net.set_params(vec)
    st = OP.adam_init()
    cur = OP.unpack(vec.astype(np.float64))
    xd, td = torch.tensor(X, device="cuda"), torch.tensor(theta, device="cuda")
    for step, lr in enumerate((1e-3, 5e-4, 2e-3)):
        net.train_step(xd, td, lr)
        g = OP.unpack(net.grads().astype(np.float64))
        cur, st = OP.adam_step(cur, g, st, lr)
        got = net.params().astype(np.float64)
        assert np.max(np.abs(got - OP.pack(cur))) <= 2e-6 * (step + 1), np.max(np.abs(got - OP.pack(cur)))
        cur = OP.unpack(got)
    net.close()


def test_training_reduces_loss():
    import torch
    B = 256
    params, vec, X, _ = _rand_problem(B, 4)
    rng = np.random.default_rng(5)
    # targets that depend on the inputs: theta = tanh(linear map of x) + noise
    Wt = rng.standard_normal((OP.N_THETA, OP.N_IN)) * 0.5
    theta = (np.tanh(X.astype(np.float64) @ Wt.T) + 0.1 * rng.standard_normal((B, OP.N_THETA))).astype(np.float32)
    net = _net(B)
    net.set_params(OP.pack(OP.init_params(0)).astype(np.float32))
    xd, td = torch.tensor(X, device="cuda"), torch.tensor(theta, device="cuda")
    losses = [float(net.train_step(xd, td, 2e-3).item()) for _ in range(300)]
    assert losses[-1] < losses[0] - 0.5, (losses[0], losses[-1])
    net.close()


def test_encoding_against_oracle():
    import torch
    from paper_1904_06680_gb300 import npp, proposal
    b = inputs.scene_proposal_batch(3, S=24, N=64, T=40, n_layouts=4)
    pl = npp.Planner(b["preset"], max_N=64, max_T=40, max_M=b["obs"].shape[0])
    obs = torch.tensor(b["obs"], dtype=torch.float32, device="cuda")
    x = proposal.encode(pl, b["scenes"], obs).cpu().numpy().astype(np.float64)
    x2 = proposal.encode(pl, b["scenes"], obs).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(x, x2)           # deterministic
    f32 = parity.f32
    for i, sc in enumerate(b["scenes"]):
        o = b["obs"][sc["obs_offset"]:sc["obs_offset"] + sc["M"]]
        xo, h, amb = OP.encode(b["preset"], f32(sc["state"]), f32(sc["goal"]), f32(o), sc["T"])
        hg = x[i, :64] / (1.0 - x[i, :64])
        assert np.all(np.abs(hg - h) <= 1e-5 * (1 + h) + amb + 1e-6), (i, np.max(np.abs(hg - h) - amb))
        np.testing.assert_allclose(x[i, 64:], xo[64:], rtol=1e-5, atol=1e-6)
    pl.close()


def _mixed_scene(seed):
    sc = inputs.tiny_scene(seed, N=3000, T=25, M=250, width=16, box=20.0)
    rng = np.random.default_rng(seed)
    mu = (rng.standard_normal(450) * 0.5).astype(np.float32)
    sd = np.exp(rng.uniform(-2, 0.5, 450)).astype(np.float32)
    return sc, mu, sd


@pytest.mark.parametrize("n_prop", [0, 1000, 3000])
def test_mixed_plan_step_against_oracle(n_prop):
    import torch
    from oracle import oracle as orc
    from paper_1904_06680_gb300 import npp
    sc, mu, sd = _mixed_scene(21)
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M, record_samples=True)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    npp.npp_plan_step_proposal(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], sc["t_index"], None,
                               torch.tensor(mu, device="cuda"), torch.tensor(sd, device="cuda"), n_prop,
                               pl.outputs())
    torch.cuda.synchronize()
    g = pl.result(N, T)
    pl.close()
    st, gl, ob, goal_ev, obs_ev = parity.oracle_inputs(sc)
    o = orc.rollout_samples(sc["preset"], sc["seed"], sc["t_index"], np.arange(N), [0, 0, 0, st[3]], st[4:6],
                            goal_ev, obs_ev, T, record=False, mu=mu, sigma=sd, n_prop=n_prop)
    w = parity.winner_check(g, o["cost"], o["first_hit"])
    assert w["agree_frac"] > 0.97, w
    assert w.get("gpu_pick_in_agree", True), w
    assert abs(w["gpu_pick_oracle_cost"] - w["best_unambiguous"]) <= parity.COST_RTOL * max(1.0, abs(w["best_unambiguous"])), w
    # the winner's parameters, regenerated by the epilogue, bit-exact
    b = g["best_idx"]
    want = orc.theta_mixed(sc["seed"], sc["t_index"], b, 450, mu, sd, n_prop)
    np.testing.assert_array_equal(g["params"], want)


def test_proposal_samples_bit_exact():
    """Every sample from the proposal: the winner is a proposal sample and
    its regenerated parameters equal the oracle's fmaf(sigma, eps, mu); the
    samples of a second step with the proposal off are the isotropic ones."""
    import torch
    from oracle import oracle as orc
    from paper_1904_06680_gb300 import npp
    sc, mu, sd = _mixed_scene(22)
    N, T = 512, sc["T"]
    M = sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    mu_d, sd_d = torch.tensor(mu, device="cuda"), torch.tensor(sd, device="cuda")
    for t_index in (5, 6, 7):
        npp.npp_plan_step_proposal(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], t_index, None,
                                   mu_d, sd_d, N, pl.outputs())
        torch.cuda.synchronize()
        r = pl.result(N, T)
        want = orc.theta_mixed(sc["seed"], t_index, r["best_idx"], 450, mu, sd, N)
        np.testing.assert_array_equal(r["params"], want)
        iso = orc.theta(sc["seed"], t_index, r["best_idx"], 450)
        assert not np.array_equal(want, iso)
    pl.close()


def test_mixed_plan_rejects_bad_arguments():
    import torch
    from paper_1904_06680_gb300 import npp
    sc, mu, sd = _mixed_scene(23)
    pl = npp.Planner(sc["preset"], max_N=100, max_T=25, max_M=250)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    for n_prop, m in [(-1, mu), (101, mu), (10, None)]:
        with pytest.raises(npp.NppError):
            npp.npp_plan_step_proposal(pl.h, sc["state"], sc["goal"], obs, 250, 100, 25, 1, 0, None,
                                       None if m is None else torch.tensor(m, device="cuda"),
                                       torch.tensor(sd, device="cuda"), n_prop, pl.outputs())
    pl.close()


def test_plain_pairs_and_training_run():
    """Pairs from the plain batched planner feed the training loop."""
    from paper_1904_06680_gb300 import proposal
    X, Th, cost = proposal.generate(0, 1024, N=1024, T=40, chunk=512)
    assert X.shape[0] > 512 and Th.shape == (X.shape[0], 450) and np.all(np.isfinite(cost))
    net = proposal.ProposalNet(batch=256)
    net.init(0)
    hist = proposal.train(net, X, Th, epochs=5, lr=1e-3)
    assert hist[-1] < hist[0], hist
    net.close()


def test_learned_proposal_gains_over_plain():
    """The training recipe, shortened (8 rounds of 4096 scenes at N = 2048),
    then held-out scenes: the mixed plan step (half proposal samples) at
    N = 512 has a clearly lower mean cost than the plain one at N = 512,
    and the proposal's samples win most scenes."""
    from paper_1904_06680_gb300 import proposal
    net, stats = proposal.train_proposal(rounds=8, S=4096, N=2048, epochs=4)
    assert stats[-1]["proposal_won"] > stats[0]["proposal_won"] + 0.08, stats
    res = proposal.evaluate(net, 1, S=96, Ns=(512,), prop_frac=0.5)[512]
    assert res["n_scenes"] > 60
    assert res["mixed"] < res["plain"] - 0.1, res
    assert res["proposal_won"] > 0.55, res
    net.close()


def test_proposal_reaches_plain_cost_at_a_quarter_of_the_samples():
    """The learned proposal's target: after the training recipe (30 rounds of
    8192 course-like scenes at N = 2048, expert iteration), on 256 held-out
    scenes the mixed plan step (half of its samples from the proposal, half
    isotropic, every sample judged by the exact rollout cost, so the plain
    sampler's samples win whenever the proposal's are worse) with N/4 = 512
    samples has a lower mean cost than the plain plan step with N = 2048
    samples, and so does N/4 = 2048 against N = 8192."""
    from paper_1904_06680_gb300 import proposal
    net, stats = proposal.train_proposal(rounds=30, S=8192, N=2048, epochs=4)
    res = proposal.evaluate(net, 2, S=256, Ns=(2048, 8192), prop_frac=0.5)
    net.close()
    for N in (2048, 8192):
        r = res[N]
        assert r["n_scenes"] > 200, r
        assert r["mixed_quarter"] <= r["plain"] - 0.02, (N, r)
