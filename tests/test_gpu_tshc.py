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
