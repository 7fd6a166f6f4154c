"""The allocation-free plan step (npp_plan_step_noalloc) against the regular
handle-based plan step.

Callers that cannot allocate device memory -- a plugin whose host
application owns all device allocations, or a real-time loop that must not
call cudaMalloc once it runs -- use npp_plan_step_noalloc, whose workspace is
a fixed static device array.  It runs the trajectory kernel and epilogue of
npp_plan_step with the shared-memory brute-force collision check (point
slices: collide_variant 3 for N <= 8192, else 4).  The regular plan step is
forced onto that same check here, so two calls in a row must reproduce its
outputs bit for bit (a layout or stale-scratch error in the static array
would show as a difference).  This file is collected last so that a run
stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

pytestmark = pytest.mark.gpu

def _run_both(sc, npp, torch):
    N, T = sc["N"], sc["T"]
    M = sc["obs"].shape[0]
    dev = torch.device("cuda", 0)
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device=dev)
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M)
    # the collision check the allocation-free entry point runs
    npp.npp_set_option(pl.h, "collide_variant", 3 if N <= 8192 else 4)
    pl.plan(sc["state"], sc["goal"], obs, N, T, sc["seed"], sc["t_index"])
    torch.cuda.synchronize()
    ref = pl.result(N, T)
    cfg = npp.make_config(sc["preset"], N, T, M)
    nt = npp.npp_n_theta(cfg)
    best = torch.zeros(8, dtype=torch.int32, device=dev)
    params = torch.zeros(nt, dtype=torch.float32, device=dev)
    controls = torch.zeros(T, 2, dtype=torch.float32, device=dev)
    traj = torch.zeros(T + 1, 4, dtype=torch.float32, device=dev)
    costs = torch.zeros(N, dtype=torch.float32, device=dev)
    fh = torch.zeros(N, dtype=torch.int32, device=dev)
    out = npp.npp_outputs()
    out.best, out.params, out.controls = best.data_ptr(), params.data_ptr(), controls.data_ptr()
    out.trajectory, out.costs, out.first_hit = traj.data_ptr(), costs.data_ptr(), fh.data_ptr()
    npp.npp_plan_step_noalloc(cfg, sc["state"], sc["goal"], obs, M, N, T, sc["seed"], sc["t_index"],
                              None, out)
    torch.cuda.synchronize()
    b = best.cpu()
    got = dict(best_idx=int(b[0]), status=int(b[1]), best_cost=b[2:3].view(torch.float32).item(),
               params=params.cpu().numpy(), controls=controls.cpu().numpy(),
               trajectory=traj.cpu().numpy(), costs=costs.cpu().numpy(), first_hit=fh.cpu().numpy())
    pl.close()
    return ref, got


def test_noalloc_matches_plan_step_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_06680_gb300 import npp
    # two calls in a row on different workloads (the second reuses the array
    # the first left behind)
    for sc in (inputs.scene_course(0), inputs.tiny_scene(41, N=777, T=23, M=97, width=16, box=30.0)):
        ref, got = _run_both(sc, npp, torch)
        assert got["best_idx"] == ref["best_idx"] and got["status"] == ref["status"]
        assert np.array_equal(got["first_hit"], ref["first_hit"])
        assert np.array_equal(got["params"], ref["params"])
        assert np.array_equal(got["costs"], ref["costs"])
        assert got["best_cost"] == ref["best_cost"] or (np.isinf(got["best_cost"]) and np.isinf(ref["best_cost"]))
        assert np.array_equal(got["controls"], ref["controls"])
        assert np.array_equal(got["trajectory"], ref["trajectory"])


def test_noalloc_rejects_oversized_request():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_06680_gb300 import npp
    sc = inputs.tiny_scene(42, N=16384, T=42, M=10, width=16)
    cfg = npp.make_config(sc["preset"], 16384, 42, 10)
    out = npp.npp_outputs()
    best = torch.zeros(8, dtype=torch.int32, device="cuda")
    out.best = best.data_ptr()
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    with pytest.raises(npp.NppError) as ei:
        npp.npp_plan_step_noalloc(cfg, sc["state"], sc["goal"], obs, 10, 16384, 42, 1, 0, None, out)
    assert ei.value.status == npp.NPP_INVALID_ARG
    assert "sample-steps" in npp.npp_last_error(None)
    with pytest.raises(npp.NppError):
        npp.npp_plan_step_noalloc(cfg, sc["state"], sc["goal"], obs, 10, 16385, 5, 1, 0, None, out)
