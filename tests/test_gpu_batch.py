"""Batched planning (npp_plan_batch): every scene of a mixed batch -- three
network widths, ragged N, T and M, a scene without obstacles, one whose
points do not fit in shared memory -- must reproduce npp_plan_step on that
scene alone."""
import numpy as np
import pytest

from paper_1904_06680_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _scenes():
    spec = [(16, 700, 20, 150), (32, 333, 33, 40), (64, 129, 12, 301), (16, 1, 5, 9),
            (32, 2048, 25, 0), (64, 65, 40, 1200), (16, 257, 17, 15001), (32, 96, 8, 77)]
    scs = []
    for i, (w, N, T, M) in enumerate(spec):
        sc = inputs.tiny_scene(50 + i, N=N, T=T, M=M, width=w, box=40.0)
        scs.append(sc)
    return scs


def test_batch_matches_single_plan_steps():
    import torch
    from paper_1904_06680_gb300 import npp
    scs = _scenes()
    p = scs[0]["preset"]                       # all scenes share the vehicle constants
    obs_all = np.concatenate([sc["obs"] for sc in scs if sc["obs"].shape[0]] + [np.zeros((0, 4))])
    offs = np.cumsum([0] + [sc["obs"].shape[0] for sc in scs])
    descs = [dict(state=sc["state"], goal=sc["goal"], N=sc["N"], T=sc["T"], M=sc["obs"].shape[0],
                  width=sc["preset"]["widths"][1], obs_offset=int(offs[i]), seed=sc["seed"],
                  t_index=sc["t_index"]) for i, sc in enumerate(scs)]
    max_N = max(d["N"] for d in descs)
    max_T = max(d["T"] for d in descs)
    max_M = max(d["M"] for d in descs)
    pl = npp.Planner(p, max_N=1, max_T=1, max_M=1)          # constants only
    scenes = npp.make_scenes(descs)
    B = npp.npp_batch_create(pl.h, scenes)
    S = len(descs)
    off = npp.npp_batch_offsets(B, S)
    dev = "cuda"
    best = torch.zeros(S * 8, dtype=torch.int32, device=dev)
    params = torch.zeros(int(off[S, 0]), dtype=torch.float32, device=dev)
    ctrl = torch.zeros(int(off[S, 1]) * 2, dtype=torch.float32, device=dev)
    traj = torch.zeros(int(off[S, 2]) * 4, dtype=torch.float32, device=dev)
    costs = torch.zeros(int(off[S, 3]), dtype=torch.float32, device=dev)
    fh = torch.zeros(int(off[S, 3]), dtype=torch.int32, device=dev)
    out = npp.npp_batch_outputs()
    out.best, out.params, out.controls = best.data_ptr(), params.data_ptr(), ctrl.data_ptr()
    out.trajectory, out.costs, out.first_hit = traj.data_ptr(), costs.data_ptr(), fh.data_ptr()
    obs_dev = torch.tensor(obs_all, dtype=torch.float32, device=dev)
    for rep in range(2):                        # twice: the work queues must reset
        npp.npp_plan_batch(B, obs_dev, out)
        torch.cuda.synchronize()
        bh = best.cpu().view(S, 8)
        for i, (sc, d) in enumerate(zip(scs, descs)):
            sp = npp.Planner(sc["preset"], max_N=d["N"], max_T=d["T"], max_M=max(1, d["M"]))
            o = torch.tensor(sc["obs"], dtype=torch.float32, device=dev) if d["M"] else None
            sp.plan(sc["state"], sc["goal"], o, d["N"], d["T"], sc["seed"], sc["t_index"])
            torch.cuda.synchronize()
            r = sp.result(d["N"], d["T"])
            sp.close()
            a, b = int(off[i, 3]), int(off[i, 3]) + d["N"]
            assert np.array_equal(fh[a:b].cpu().numpy(), r["first_hit"]), i
            assert np.array_equal(costs[a:b].cpu().numpy(), r["costs"]), i
            assert int(bh[i, 0]) == r["best_idx"] and int(bh[i, 1]) == r["status"], i
            nt = 12 * d["width"] + d["width"] ** 2 + 2
            assert np.array_equal(params[int(off[i, 0]):int(off[i, 0]) + nt].cpu().numpy(), r["params"]), i
            c = ctrl[2 * int(off[i, 1]):2 * (int(off[i, 1]) + d["T"])].cpu().numpy().reshape(-1, 2)
            np.testing.assert_allclose(c, r["controls"], rtol=1e-6, atol=1e-6)
            t = traj[4 * int(off[i, 2]):4 * (int(off[i, 2]) + d["T"] + 1)].cpu().numpy().reshape(-1, 4)
            np.testing.assert_allclose(t, r["trajectory"], rtol=1e-6, atol=1e-4)
    npp.npp_batch_destroy(B)
    pl.close()


def test_batch_options_and_graph_replay_identical():
    """Every collision check and launch shape the autotuner may pick (binned
    and brute force), and a CUDA-graph capture of the batch replayed twice,
    give the same results."""
    import torch
    from paper_1904_06680_gb300 import autotune, npp
    b = inputs.scene_batch(5, S=24, N_range=(64, 2048), M_range=(20, 3000), T_range=(5, 30))
    pl = npp.Planner(b["preset"], max_N=1, max_T=1, max_M=1)
    scenes = npp.make_scenes(b["scenes"])
    S = len(b["scenes"])
    B = npp.npp_batch_create(pl.h, scenes)
    off = npp.npp_batch_offsets(B, S)
    best = torch.zeros(S * 8, dtype=torch.int32, device="cuda")
    costs = torch.zeros(int(off[S, 3]), dtype=torch.float32, device="cuda")
    fh = torch.zeros(int(off[S, 3]), dtype=torch.int32, device="cuda")
    params = torch.zeros(int(off[S, 0]), dtype=torch.float32, device="cuda")
    out = npp.npp_batch_outputs()
    out.best, out.costs, out.first_hit, out.params = best.data_ptr(), costs.data_ptr(), fh.data_ptr(), params.data_ptr()
    obs = torch.tensor(b["obs"], dtype=torch.float32, device="cuda")

    def snap():
        torch.cuda.synchronize()
        return best.cpu().clone(), costs.cpu().clone(), fh.cpu().clone(), params.cpu().clone()

    npp.npp_plan_batch(B, obs, out)
    ref = snap()
    assert 0 < int((ref[2] >= 0).sum()) < ref[2].numel()
    for cand in autotune.BATCH_CANDIDATES:
        autotune._set_batch(B, cand)
        for t in (best, costs, fh, params):
            t.zero_()
        npp.npp_plan_batch(B, obs, out)
        got = snap()
        for a, r in zip(got, ref):
            assert torch.equal(a, r), cand
    choice, ms = autotune.tune_batch(B, obs, out, key="test24", reps=1)
    assert tuple(choice) in autotune.BATCH_CANDIDATES and len(ms) == len(autotune.BATCH_CANDIDATES)
    # capture in a CUDA graph on a side stream, replay twice
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        npp.npp_plan_batch(B, obs, out, stream=torch.cuda.current_stream())
    for _ in range(2):
        for t in (best, costs, fh, params):
            t.zero_()
        g.replay()
        got = snap()
        for a, r in zip(got, ref):
            assert torch.equal(a, r)
    with pytest.raises(npp.NppError):
        npp.npp_batch_set_option(B, "slices", 3)
    with pytest.raises(npp.NppError):
        npp.npp_batch_set_option(B, "collide", 2)
    npp.npp_batch_destroy(B)
    pl.close()
