"""Host-side pieces of the benchmark that decide reported outcomes, checked
on the CPU: the collision check of executed poses (mission success) against
the oracle's point-in-rectangle test, and the algorithmic-work counts."""
import os

import numpy as np

import bench
from paper_1904_06680_gb300 import inputs


def test_executed_collisions_match_oracle(orc):
    p = inputs.planner(32)
    rng = np.random.default_rng(3)
    obs = np.zeros((40, 4))
    obs[:, :2] = rng.uniform(-10, 10, (40, 2))
    obs[:15, 2:] = rng.uniform(-1, 1, (15, 2))
    log = np.zeros((60, 8), np.float32)
    log[:, 0] = rng.uniform(-6, 6, 60)
    log[:, 1] = rng.uniform(-6, 6, 60)
    log[:, 2] = rng.uniform(-3, 3, 60)
    got = bench.executed_collisions(log, obs, p)
    want = [t for t in range(60)
            if orc.collide(p, float(log[t, 0]), float(log[t, 1]), float(log[t, 2]), obs, tau=t * p["Ts"])[0]]
    assert got == want
    assert 0 < len(want) < 60


def test_algorithmic_work_counts():
    fh = np.array([-1, 0, 5, 39])
    T, M, W = 40, 100, 32
    fma_c, fma_t, checks = bench.algorithmic_work(fh, T, M, W)
    live_states = (T + 1) + 1 + 6 + 40          # states 0..first_hit (all T+1 if free)
    assert checks == live_states * M
    assert fma_c == 4.0 * checks
    assert fma_t == (T + 0 + 5 + 39) * (W * W + 10 * W)


def test_profiled_traffic_entries_are_current():
    """Every DRAM-traffic entry in profiles/traffic.json names a kernel whose
    CUDA sources are known and unchanged since the capture (an entry whose
    kernel changed would report counters of other code); the per-workload
    entries of kernels used by several workloads are found by workload."""
    import json
    import bench
    rec = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    assert rec["kernels"]
    for key, ent in rec["kernels"].items():
        name = key.split("@")[0]
        assert bench.kernel_sources_hash(name) is not None, key
        assert ent["sources"] == bench.kernel_sources_hash(name), key
        assert ent["dram_bytes_per_launch"] == ent["read"] + ent["write"], key
        assert "--clock-control none" in ent["command"], key
    for key in rec["kernels"]:
        if "@" in key:
            name, wl = key.split("@")
            assert bench.profiled_traffic(name, wl) == rec["kernels"][key]["dram_bytes_per_launch"]


def test_grid_bytes_counts_reads_and_writes():
    """Per grid: M points read in the count and the scatter pass (16 B
    each), 128 x 128 + 1 cell starts and M sorted points (8 B) written."""
    import bench
    assert bench.grid_bytes(0, 0) == 4.0 * (128 * 128 + 1)
    assert bench.grid_bytes(0, 10) == 10 * 16 * 2 + 4.0 * (128 * 128 + 1) + 10 * 8
    assert bench.grid_bytes(100, 8192) == 101 * (8192 * 40 + 4.0 * 16385)


def test_automatic_brute_force_variant_names():
    """The bench names the kernel the library's automatic brute-force choice
    runs: for N >= 6144 variant 2 up to 1200 points, else 4; for fewer
    samples 1 from 6000 points, 2 up to 64 points, else 3 (the rule the
    library documents for collide_variant -1 below its binning threshold)."""
    import bench
    cases = {(20, 20480): 2, (157, 16384): 2, (1200, 8192): 2, (1201, 8192): 4, (20, 4096): 2, (64, 1024): 2,
             (65, 1024): 3, (157, 4096): 3, (5999, 2048): 3, (6000, 2048): 1, (8000, 990): 1}
    for (M, N), v in cases.items():
        assert bench.brute_auto(M, N) == v, (M, N)
