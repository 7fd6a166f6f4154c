"""The host-buffer plan step (npp_plan_step_host: obstacle and warm-start
copies in, the plan step on the handle's stream, the outputs copied back,
synchronised) against the device-buffer plan step on the same handle
settings: the same winner, summary, parameters, controls, trajectory and
per-sample costs and first collisions, bit for bit -- the entry point behind
the benchmark's end-to-end figure."""
import ctypes

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _host_plan(pl, sc, warm, npp, torch):
    N, T = sc["N"], sc["T"]
    hb = npp.npp_best()
    params = torch.zeros(pl.n_theta, dtype=torch.float32).pin_memory()
    ctrl = torch.zeros(T, 2, dtype=torch.float32).pin_memory()
    traj = torch.zeros(T + 1, 4, dtype=torch.float32).pin_memory()
    costs = np.zeros(N, np.float32)                      # pageable host memory works as well
    fh = np.zeros(N, np.int32)
    o = npp.npp_outputs()
    o.best = ctypes.addressof(hb)
    o.params, o.controls, o.trajectory = params.data_ptr(), ctrl.data_ptr(), traj.data_ptr()
    o.costs, o.first_hit = costs.ctypes.data, fh.ctypes.data
    obs = torch.tensor(sc["obs"], dtype=torch.float32).pin_memory()
    w = None if warm is None else torch.tensor(warm, dtype=torch.float32).pin_memory()
    npp.npp_plan_step_host(pl.h, sc["state"], sc["goal"], obs, obs.shape[0], N, T, sc["seed"], sc["t_index"], w, o)
    return dict(best_idx=hb.best_idx, status=hb.status, best_cost=hb.best_cost, first_hit_best=hb.first_hit,
                params=params.numpy().copy(), controls=ctrl.numpy().copy(), trajectory=traj.numpy().copy(),
                costs=costs, first_hit=fh)


# course scenes (2000 points) under a brute-force check (option 3), the
# automatic two-kernel binned check (width 32) and the automatic windowed
# check inside the trajectory kernel (width 64)
@pytest.mark.parametrize("width,N,seed,variant", [(32, 2048, 1, 3), (32, 4096, 2, -1), (64, 4096, 3, -1)])
@pytest.mark.parametrize("use_warm", [False, True])
def test_host_entry_equals_device_entry(width, N, seed, variant, use_warm):
    import torch
    from paper_1904_06680_gb300 import npp
    sc = inputs.scene_course(seed, N=N, width=width)
    T, M = sc["T"], sc["obs"].shape[0]
    pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M)
    npp.npp_set_option(pl.h, "collide_variant", variant)
    warm = None
    if use_warm:
        warm = (np.random.default_rng(seed).standard_normal(pl.n_theta) * 0.5).astype(np.float32)
    w_dev = None if warm is None else torch.tensor(warm, device="cuda")
    pl.plan(sc["state"], sc["goal"], torch.tensor(sc["obs"], dtype=torch.float32, device="cuda"), N, T,
            sc["seed"], sc["t_index"], warm=w_dev)
    torch.cuda.synchronize()
    dev = pl.result(N, T)
    host = _host_plan(pl, sc, warm, npp, torch)
    pl.close()
    assert (host["best_idx"], host["status"], host["first_hit_best"]) == \
        (dev["best_idx"], dev["status"], dev["first_hit_best"])
    assert np.float32(host["best_cost"]).view(np.int32) == np.float32(dev["best_cost"]).view(np.int32)
    for k in ("params", "controls", "trajectory", "first_hit"):
        assert np.array_equal(host[k], dev[k]), k
    assert np.array_equal(host["costs"].view(np.int32), dev["costs"].view(np.int32))
    assert 0 < np.sum(dev["first_hit"] >= 0) < N
