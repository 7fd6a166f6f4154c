"""The hill climb's restart loop on the device (npp_plan_tshc) against the
oracle's loop: the winner after every number of rounds, its cost and its
parameters (bit-exact), and the non-increasing best cost."""
import os
import sys

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
import parity  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tshc_against_oracle():
    import torch
    from oracle import oracle as orc
    from paper_1904_06680_gb300 import npp
    sc = inputs.tiny_scene(23, N=1024, T=20, M=150, width=16, box=16.0)
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    st, gl, ob = (parity.f32(sc[k]) for k in ("state", "goal", "obs"))
    costs = []
    for R in (1, 2, 4):
        npp.npp_plan_tshc(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], sc["t_index"], None, R, 0.25,
                          pl.outputs())
        torch.cuda.synchronize()
        g = pl.result(N, T)
        o = orc.plan_tshc(sc["preset"], st, gl, ob.reshape(-1, 4), N, T, sc["seed"], sc["t_index"], R, 0.25)
        assert g["status"] == 0 and o["status"] == 0
        assert abs(g["best_cost"] - o["best_cost"]) <= parity.COST_RTOL * max(1.0, abs(o["best_cost"])), (R, g["best_cost"], o["best_cost"])
        assert g["best_idx"] == o["best_idx"], R
        np.testing.assert_array_equal(g["params"], o["best_theta"].astype(np.float32))
        costs.append(g["best_cost"])
    assert costs[1] <= costs[0] and costs[2] <= costs[1]
    with pytest.raises(npp.NppError):
        npp.npp_plan_tshc(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], 0, None, 0, 0.25, pl.outputs())
    with pytest.raises(npp.NppError):
        npp.npp_plan_tshc(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], 0, None, 2, -1.0, pl.outputs())
    pl.close()


def test_loop_restarts_equal_plan_tshc():
    """A closed loop with restart rounds (npp_set_loop_restarts) runs, at its
    first sampling time, the same rounds as npp_plan_tshc: the same winner,
    cost, first control and per-sample costs of the last round; invalid
    settings are refused."""
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.tiny_scene(24, N=1024, T=20, M=150, width=16, box=16.0)
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    R, sigma = 4, 0.25
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    npp.npp_plan_tshc(pl.h, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], 0, None, R, sigma, pl.outputs())
    torch.cuda.synchronize()
    g = pl.result(N, T)
    npp.npp_set_loop_restarts(pl.h, R, sigma)
    L = npp.npp_loop_create(pl.h, sc["state"], [sc["goal"]], inputs.EPS, obs, M, N, T, sc["seed"], max_log=8)
    npp.npp_loop_run(L, 1)
    st = npp.npp_loop_read(L)
    costs, fh = npp.npp_loop_samples(L, N)
    log = npp.npp_loop_log(L, 8)
    npp.npp_loop_destroy(L)
    assert st["best_idx"] == g["best_idx"] and st["status"] == g["status"]
    assert np.float32(st["best_cost"]) == np.float32(g["best_cost"])
    np.testing.assert_array_equal(log[0, 4:6], g["controls"][0])
    np.testing.assert_array_equal(costs, g["costs"])
    np.testing.assert_array_equal(fh, g["first_hit"])
    with pytest.raises(npp.NppError):
        npp.npp_set_loop_restarts(pl.h, 0, sigma)
    with pytest.raises(npp.NppError):
        npp.npp_set_loop_restarts(pl.h, 3, 0.0)
    npp.npp_set_loop_restarts(pl.h, 1)
    pl.close()
