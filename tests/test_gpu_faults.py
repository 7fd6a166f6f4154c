"""Failure detection without a GPU fault: the library's bounded device wait
gives up on a barrier that nothing completes, and the context stays usable;
a fault flag set from the host, as a timed-out wait of a plan step's kernels
sets it, comes back as NPP_DEVICE_TIMEOUT in that step's result, once."""
import ctypes
import time

import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(pl, sc):
    import torch
    obs = torch.tensor(sc["obs"], dtype=torch.float32, device="cuda")
    pl.plan(sc["state"], sc["goal"], obs, sc["N"], sc["T"], sc["seed"], sc["t_index"])
    torch.cuda.synchronize()
    return pl.result(sc["N"], sc["T"])


def test_bounded_wait_gives_up_and_context_stays_usable():
    from paper_1904_06680_gb300 import npp
    assert npp.npp_wait_probe(1_000_000, True)
    t0 = time.perf_counter()
    assert not npp.npp_wait_probe(2_000_000, False)      # ~1 ms of clock, nothing arrives
    assert time.perf_counter() - t0 < 5.0
    for bad in ((0, True), (5_000_000_000, False)):
        with pytest.raises(npp.NppError):
            npp.npp_wait_probe(*bad)
    # the context is intact: a plan step with the brute-force staging runs
    sc = inputs.tiny_scene(3, 400, 12, 300, width=16)
    pl = npp.Planner(sc["preset"], max_N=sc["N"], max_T=sc["T"], max_M=300)
    npp.npp_set_option(pl.h, "collide_variant", 3)
    r = _plan(pl, sc)
    pl.close()
    assert r["status"] in (npp.NPP_OK, npp.NPP_INFEASIBLE)


def test_injected_fault_reported_once():
    from paper_1904_06680_gb300 import npp
    sc = inputs.tiny_scene(4, 500, 15, 200, width=16)
    pl = npp.Planner(sc["preset"], max_N=sc["N"], max_T=sc["T"], max_M=200)
    ok = _plan(pl, sc)
    assert ok["status"] in (npp.NPP_OK, npp.NPP_INFEASIBLE)
    npp.npp_inject_fault(pl.h)
    assert _plan(pl, sc)["status"] == npp.NPP_DEVICE_TIMEOUT
    again = _plan(pl, sc)                                # the flag was cleared
    assert again["status"] == ok["status"] and again["best_idx"] == ok["best_idx"]
    # the host-buffer entry point returns the status
    import torch
    hb = npp.npp_best()
    o = npp.npp_outputs()
    o.best = ctypes.addressof(hb)
    obs = torch.tensor(sc["obs"], dtype=torch.float32).pin_memory()
    npp.npp_inject_fault(pl.h)
    with pytest.raises(npp.NppError) as ei:
        npp.npp_plan_step_host(pl.h, sc["state"], sc["goal"], obs, obs.shape[0], sc["N"], sc["T"], sc["seed"],
                               sc["t_index"], None, o)
    assert ei.value.status == npp.NPP_DEVICE_TIMEOUT
    npp.npp_plan_step_host(pl.h, sc["state"], sc["goal"], obs, obs.shape[0], sc["N"], sc["T"], sc["seed"],
                           sc["t_index"], None, o)
    assert hb.status in (npp.NPP_OK, npp.NPP_INFEASIBLE)
    pl.close()
