"""Multi-process host logic on CPU (gloo, world size 2): the bench's rank to
scene mapping, max-over-ranks timing and whole-job rate, and the min-merge
of packed best keys of a sample-sharded plan, checked against the oracle's
single-process winner."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1904_06680_gb300 import inputs, multi
        from oracle import oracle as orc
        r, w, loc = multi.dist_env()
        res = {"env": (r, w, loc), "seed": multi.rank_seed(7, r)}
        res["max"] = multi.max_over_ranks([1.0 + r, 10.0 - r, 3.5])
        res["rate"] = multi.whole_job_rate(1000, w, res["max"][0])
        # sample-sharded plan of one scene: each rank rolls out its index range
        sc = inputs.tiny_scene(3, N=96, T=15, M=60, width=16, box=12.0)
        st = np.asarray(sc["state"], np.float32).astype(np.float64)
        gl = np.asarray(sc["goal"], np.float32).astype(np.float64)
        ob = np.asarray(sc["obs"], np.float32).astype(np.float64)
        goal_ev, obs_ev = orc.frame_to_ev(st, gl, ob)
        n0, cnt = multi.shard(sc["N"], w, r)
        idx = np.arange(n0, n0 + cnt, dtype=np.int32)
        o = orc.rollout_samples(sc["preset"], sc["seed"], sc["t_index"], idx, [0, 0, 0, st[3]], st[4:6], goal_ev,
                                obs_ev, sc["T"], record=False)
        keys = []
        for n, c, fh in zip(idx, o["cost"], o["first_hit"]):
            if fh < 0:
                keys.append((int(np.float32(c).view(np.uint32)) << 32) | int(n))
            else:
                keys.append((1 << 63) | ((sc["T"] - int(fh)) << 32) | int(n))
        res["shard"] = (n0, cnt)
        res["key"] = multi.min_key(min(keys))
        out.put((r, res))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0]["env"] == (0, 2, 0) and got[1]["env"] == (1, 2, 1)
    assert got[0]["seed"] != got[1]["seed"]
    for r in range(world):
        assert got[r]["max"] == [2.0, 10.0, 3.5]
        assert got[r]["rate"] == pytest.approx(2000 / 2.0)
    # shards cover 0..N-1 exactly once
    (a0, ac), (b0, bc) = got[0]["shard"], got[1]["shard"]
    assert a0 == 0 and b0 == ac and ac + bc == 96
    # the merged key is the same on both ranks and decodes to the oracle's
    # single-process winner
    assert got[0]["key"] == got[1]["key"]
    from oracle import oracle as orc
    from paper_1904_06680_gb300 import inputs
    sc = inputs.tiny_scene(3, N=96, T=15, M=60, width=16, box=12.0)
    r = orc.plan(sc["preset"], np.asarray(sc["state"], np.float32), np.asarray(sc["goal"], np.float32),
                 np.asarray(sc["obs"], np.float32), sc["N"], sc["T"], sc["seed"], sc["t_index"])
    assert (got[0]["key"] & 0xffffffff) == r["best_idx"]
    assert (got[0]["key"] >> 63) == (1 if r["status"] != 0 else 0)


def test_single_process_identities():
    from paper_1904_06680_gb300 import multi
    assert multi.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    assert multi.min_key(12345) == 12345
    for n, w in [(10, 3), (96, 2), (7, 7), (5, 8)]:
        ranges = [multi.shard(n, w, r) for r in range(w)]
        assert sum(c for _, c in ranges) == n
        assert all(ranges[i][0] + ranges[i][1] == ranges[i + 1][0] for i in range(w - 1))
    for k in [0, 1, (1 << 63) - 1, 1 << 63, (1 << 64) - 1, (1 << 63) | 12]:
        assert multi._from_signed(multi._to_signed(k)) == k
    ks = sorted([0, 5, (1 << 63) - 1, 1 << 63, (1 << 64) - 1])
    assert [multi._to_signed(k) for k in ks] == sorted(multi._to_signed(k) for k in ks)
