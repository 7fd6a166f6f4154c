#!/usr/bin/env python
"""Planner benchmark: rollout-steps/s of the closed-loop plan step.

Default workload (one GPU, the largest single-GPU configuration): the large
closed loop, N = 65536 sampled 8-64-64-2 networks per plan step, horizon
T = 100, M = 8192 obstacle points (20 % on moving car outlines) in an
80 x 80 m area, per-step spatial binning of the points.  A "step" is one
sampling time of the closed loop run on the device as one CUDA-graph
replay: sampling, rollout, collision checks (at width 64 window by window
inside the trajectory kernel), selection, winner epilogue, then the
simulated vehicle, obstacle and waypoint advance; the winner's parameters
warm-start the next step.  `--workload course` runs the forward/reverse
waypoint course (N = 16384, T = 40, 8-32-32-2, M = 2000); batch, proposal
and mission are the other workloads.

value   = N * T * K / (sum of the K steps' device time), inputs resident in
          HBM, L2 flushed (256 MiB write) between steps, CUDA events captured
          in the step graph;
e2e     = the same closed loop through the host-buffer entry point (obstacle
          copy in, plan, result copy out, synchronise, host vehicle model),
          wall clock per plan call;
roofline = the dominant kernel (the trajectory kernel, with the windowed
          check at width 64): algorithmic FP32 FMAs (W^2 + 10 W per control
          step of a sample up to its first collision) over its event-timed
          duration, against the FMA peak SMs x 128 lanes x the maximum SM
          clock (read from the device); with a brute-force check chosen
          (--set collide_variant=0..4) the collision kernel, 4 FMAs per
          point check of a live sample; `traffic` comes from the committed
          ncu summary while the kernel sources are unchanged.

`--impl reference` times the CPU oracle on the host cores on the same
workload with a bounded number of samples per step.
Multi-GPU (torchrun): every rank plans its own scene (weak scaling, no
collective on the data path); max over ranks.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rollout-steps/s (N×T incl. M-point checks)"
UNIT = "rollout-steps/s"
DEFAULT_FUSE = -1                # the library's default of the "fuse" option (-1: at width 64)
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (4 schedulers x 32) on sm_100-class parts
SM_MAX_MHZ_NOMINAL = 2070.0      # GB300 maximum SM clock, used only when the device does not report it
BIN_DIM = 128                    # cells per side of the library's per-step grids (the grid build's table size)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="npp", choices=["npp", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="large",
                    choices=["course", "large", "batch", "proposal", "mission", "paper"],
                    help="large (default, the largest single-GPU configuration): N=65536, T=100, "
                         "8-64-64-2, 8192 points over 80x80 m with per-step spatial binning; "
                         "course: the closed-loop forward/reverse course (N=16384, T=40, 8-32-32-2, M=2000); "
                         "batch: 512 parking scenes of uneven N, T, M and width in one "
                         "graph-captured batch; proposal: the learned sampling proposal "
                         "(tensor-core GEMM roofline, training throughput, plan quality); paper: the "
                         "paper's Step-5 setting (15 restarts x 20480 samples x H=200) beside its tau_a")
    ap.add_argument("--rounds", type=int, default=30, help="proposal workload: training rounds")
    ap.add_argument("--missions", type=int, default=10, help="mission workload: scene seeds")
    ap.add_argument("--set", action="append", default=[], metavar="NAME=VALUE",
                    help="course/large: a launch option of the planner handle (npp_set_option), e.g. "
                         "collide_variant=3 or fuse=0; repeatable")
    ap.add_argument("--footprint", default="rect", choices=["rect", "car"],
                    help="course/large: the rectangle, or a two-piece car outline (general polygon check)")
    return ap.parse_args()


def dist_env():
    from paper_1904_06680_gb300 import multi
    return multi.dist_env()


class Nvml:
    """Read-only NVML queries through ctypes (clocks, clock-event reasons,
    power) for the device torch calls `cuda_index`; None-valued when the
    library or the device cannot be found."""

    # clock-event reason bits of NVML
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        import ctypes
        self.h = None
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            import torch
            pr = torch.cuda.get_device_properties(cuda_index)
            dom, bus, devn = (getattr(pr, k, None) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id"))
            h = ctypes.c_void_p()
            if bus is not None:
                bid = ("%08X:%02X:%02X.0" % (dom or 0, bus, devn or 0)).encode()
                if self.lib.nvmlDeviceGetHandleByPciBusId_v2(bid, ctypes.byref(h)) != 0:
                    h = ctypes.c_void_p()
            if not h.value and self.lib.nvmlDeviceGetHandleByIndex_v2(int(cuda_index), ctypes.byref(h)) != 0:
                return
            self.h = h
            self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(self.lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        except (OSError, AttributeError):
            self.h = None

    def _u(self, fn, *args):
        import ctypes
        v = ctypes.c_uint()
        return v.value if fn(self.h, *args, ctypes.byref(v)) == 0 else None

    def max_sm_mhz(self):
        return None if self.h is None else self._u(self.lib.nvmlDeviceGetMaxClockInfo, 1)

    def sample(self):
        """(sm MHz, reason bits, power W) now."""
        import ctypes
        mhz = self._u(self.lib.nvmlDeviceGetClockInfo, 1)
        r = ctypes.c_ulonglong()
        bits = r.value if self.reasons_fn(self.h, ctypes.byref(r)) == 0 else 0
        mw = self._u(self.lib.nvmlDeviceGetPowerUsage)
        return mhz, bits, (mw or 0) / 1000.0


def fp32_peak(cuda_index):
    """Derived FP32 FMA peak (FMA/s) of the device: SM count from the device
    properties x 128 FMA lanes x the maximum SM clock (NVML, else the
    device attribute, else the GB300 nominal), with its basis."""
    import torch
    pr = torch.cuda.get_device_properties(cuda_index)
    sms = pr.multi_processor_count
    mhz, src = Nvml(cuda_index).max_sm_mhz(), "NVML max SM clock"
    if not mhz:
        khz = getattr(pr, "clock_rate", 0) or 0
        mhz, src = (khz / 1000.0, "device clock-rate attribute") if khz else (SM_MAX_MHZ_NOMINAL, "GB300 nominal")
    return sms * FP32_LANES_PER_SM * mhz * 1e6, "derived: %d SMs x %d FP32 FMA lanes x %.0f MHz (%s)" % (
        sms, FP32_LANES_PER_SM, mhz, src)


class Clocks:
    """SM clock and throttle reasons during the timed region: an in-process
    NVML sampler (every 2 ms) plus nvidia-smi queried back to back, both on
    background threads."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.nv = []
        self.stop_flag = False
        self.thread = None
        self.nv_thread = None
        self.nvml = Nvml(gpu_index)

    def _poll_nvml(self):
        while not self.stop_flag:
            self.nv.append(self.nvml.sample())
            time.sleep(0.002)

    def _poll(self):
        while not self.stop_flag:
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout
            except (OSError, subprocess.TimeoutExpired):
                return
            for line in out.splitlines():
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    self.rows.append(parts)

    def start(self):
        import threading
        self.stop_flag = False
        self.thread = threading.Thread(target=self._poll, daemon=True)
        self.thread.start()
        if self.nvml.h is not None:
            self.nv_thread = threading.Thread(target=self._poll_nvml, daemon=True)
            self.nv_thread.start()

    def stop(self):
        self.stop_flag = True
        for t in (self.thread, self.nv_thread):
            if t is not None:
                t.join(timeout=10)
        rows = self.rows
        nv = [x for x in self.nv if x[0]]
        if nv:
            reasons = set()
            for _, bits, _ in nv:
                for b, name in Nvml.REASONS.items():
                    if bits & b:
                        reasons.add(name)
            for r in rows:
                for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                      "sw_power_cap"], r[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
            return {"sm_mhz": float(np.median([x[0] for x in nv])),
                    "sm_max_mhz": float(self.nvml.max_sm_mhz() or np.nan),
                    "sm_mhz_min": float(np.min([x[0] for x in nv])),
                    "power_w_max": float(np.max([x[2] for x in nv])),
                    "samples": len(nv), "samples_nvidia_smi": len(rows), "source": "NVML every 2 ms + nvidia-smi",
                    "reasons": sorted(reasons)}
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.nanmedian([num(r[1]) for r in rows])),
                "sm_max_mhz": float(np.nanmax([num(r[2]) for r in rows])),
                "power_w_max": float(np.nanmax([num(r[3]) for r in rows])), "samples": len(rows),
                "reasons": sorted(reasons)}


COURSE_DESC = ("closed-loop forward/reverse waypoint course: N=16384 samples, T=40, MLP 8-32-32-2, "
               "M=2000 points (500 moving), one plan step per sampling time")
LARGE_DESC = ("closed loop in an 80x80 m area: N=65536 samples, T=100, MLP 8-64-64-2, M=8192 points "
              "(20% moving, |v|<=5 m/s), per-step spatial binning of the points, one plan step per "
              "sampling time")


def workload_setup(name, seed):
    """(scene, description) of a closed-loop workload."""
    from paper_1904_06680_gb300 import inputs
    if name == "large":
        return inputs.scene_large(seed=seed), LARGE_DESC
    return inputs.scene_course(seed=seed), COURSE_DESC


def brute_auto(M, N):
    """The library's automatic brute-force collision variant (the same rule
    as its brute_auto), to name the kernel that ran."""
    if N >= 6144:
        return 2 if M <= 1200 else 4
    if M >= 6000:
        return 1
    return 2 if M <= 64 else 3


def grid_bytes(T, M):
    """Algorithmic bytes of one plan step's per-step grids: for each of the
    T + 1 grids the M world points read twice (count and scatter passes,
    16 B each), the cell-start table (BIN_DIM^2 + 1 entries of 4 B) and the
    M sorted points (8 B each) written."""
    return (T + 1) * (32.0 * M + 4.0 * (BIN_DIM * BIN_DIM + 1) + 8.0 * M)


def algorithmic_work(first_hit, T, M, W):
    """Algorithmic FP32 FMAs, split by kernel: the collision check needs 4
    per point-check of a live sample (two rows of the rotated inequality
    test); the control step needs W^2 + 10 W multiply-adds per live step
    (the MLP).  Also returns the live point-checks."""
    fh = np.asarray(first_hit)
    checks = float(np.where(fh < 0, T + 1, fh + 1).sum()) * M
    ctrl = float(np.where(fh < 0, T, fh).sum())
    return 4.0 * checks, ctrl * (W * W + 10 * W), checks


# source files whose code each profiled kernel is built from
_ROLLOUT = ("npp_rollout.cuh", "npp_device.cuh", "npp_async.cuh")
KERNEL_SOURCES = tuple(
    (kind + "<%d" % w, _ROLLOUT + ("npp_rollout_w%d.cu" % w,))      # each width's own translation unit
    for kind in ("traj_kernel", "fused_kernel") for w in (16, 32, 64)) + (
    ("bin_build_kernel", ("npp_binned.cu", "npp_rollout.cuh", "npp_device.cuh", "npp_async.cuh")),
    ("collide_binned_kernel", ("npp_binned.cu", "npp_rollout.cuh", "npp_device.cuh", "npp_async.cuh")),
    ("collide_poly_kernel", ("npp_poly.cu", "npp_rollout.cuh", "npp_device.cuh", "npp_async.cuh")),
    ("collide_", ("npp_rollout.cuh", "npp_device.cuh", "npp_collide.cu", "npp_async.cuh")),
    ("gemm_kernel", ("npp_gemm.cu", "npp_gemm.cuh", "npp_async.cuh")),
)


def kernel_sources_hash(kernel):
    """Hash of the CUDA sources a kernel is built from: its profile counters
    apply only to this code."""
    import hashlib
    d = os.path.join(ROOT, "paper_1904_06680_gb300", "csrc")
    files = next((v for k, v in KERNEL_SOURCES if kernel.startswith(k)), None)
    if files is None:
        return None
    h = hashlib.sha1()
    for f in files:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload=None):
    """DRAM bytes per launch of `kernel` from profiles/traffic.json (the entry
    "kernel@workload" where the traffic depends on the workload), or None
    when its sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    k = kernel.replace(" ", "")
    ents = {kk.replace(" ", ""): v for kk, v in rec.get("kernels", {}).items()}
    ent = ents.get("%s@%s" % (k, workload)) or ents.get(k)
    if not ent or ent.get("sources") != kernel_sources_hash(k):
        return None
    return ent.get("dram_bytes_per_launch")


def cpu_baseline(sc, state, goal, obs, T, workload, target_cpu_s=15.0):
    """Oracle (as it stands) on the host cores: a bounded sample of the first
    plan step's workload -- blocks of 1024 samples (indices 0..1024 r - 1;
    beyond N they are further Philox draws of the same distribution), each
    over the full horizon, r chosen for about `target_cpu_s` seconds of
    single-core work -- and the first 1024 samples on one core."""
    from oracle import oracle as orc
    p = sc["preset"]
    cores = os.cpu_count() or 1
    goal_ev, obs_ev = orc.frame_to_ev(state, goal, obs)
    z0 = [0.0, 0.0, 0.0, state[3]]
    probe = np.arange(1024, dtype=np.int32)
    t0 = time.perf_counter()
    orc.rollout_samples(p, sc["seed"], 0, probe, z0, state[4:6], goal_ev, obs_ev, T, n_threads=1,
                        record=False)
    single_s = max(time.perf_counter() - t0, 1e-6)
    r = int(min(64, max(1, round(target_cpu_s / single_s))))
    K = 1024 * r
    idx = np.arange(K, dtype=np.int32)
    t0 = time.perf_counter()
    orc.rollout_samples(p, sc["seed"], 0, idx, z0, state[4:6], goal_ev, obs_ev, T, n_threads=cores,
                        record=False)
    wall = time.perf_counter() - t0
    return {"value": K * T / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread": 1024 * T / single_s,
            "sample": "first plan step of the %s scene: %d x 1024 samples (the step draws %d) over "
                      "the full horizon T=%d, M=%d points (brute force), FP64 C with OpenMP on %d "
                      "threads (%.1f s wall); single_thread: the first 1024 samples on one core (%.1f s)" % (
                          workload, r, sc["N"], T, obs.shape[0], cores, wall, single_s)}


def run_npp(args):
    import torch
    from paper_1904_06680_gb300 import closed_loop, inputs, npp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)              # before the process group: NCCL binds the current device
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    sc, desc = workload_setup(args.workload, args.seed + rank)
    poly = args.footprint == "car"
    if poly:
        sc["preset"] = dict(sc["preset"], footprint=inputs.CAR_FOOTPRINT)
        desc += "; footprint: car outline with a pointed nose and a tow bar (two convex pieces, 10 faces)"
    p = sc["preset"]
    N, T = sc["N"], sc["T"]
    W = p["widths"][1]
    M = sc["obs"].shape[0]
    K, Wu = args.steps, args.warmup
    pl = npp.Planner(p, max_N=N, max_T=T, max_M=M, device=local)
    npp.npp_set_timing(pl.h, True)
    options = dict(kv.split("=", 1) for kv in args.set)
    for name, val in options.items():
        npp.npp_set_option(pl.h, name, int(val))
    obs0_dev = torch.tensor(sc["obs"], dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def device_loop_pass(nsteps: int, record: bool):
        """The closed loop on the device: one CUDA-graph replay per sampling
        time (plan step + vehicle/obstacle/waypoint advance), L2 flushed
        between replays outside the timed region."""
        L = npp.npp_loop_create(pl.h, sc["state"], sc["waypoints"], inputs.EPS, obs0_dev, M, N, T,
                                sc["seed"], max_log=max(nsteps, 1))
        out = dict(step_ms=[], collide_ms=[], traj_ms=[], fma_c=0.0, fma_t=0.0, checks=0.0,
                   free=[], best_cost=[], cand_tests=0.0, states=0.0, rolled=0.0)
        for t in range(nsteps):
            flush.zero_()
            torch.cuda.synchronize()
            npp.npp_loop_run(L, 1)
            tm = npp.npp_loop_last_timing(L)
            if record:
                ct, cs, cr = npp.npp_last_counts(pl.h)
                out["cand_tests"] += ct
                out["states"] += cs
                out["rolled"] += cr
                _, fh = npp.npp_loop_samples(L, N)
                out["step_ms"].append(tm["total"])
                out["collide_ms"].append(tm["collide"])
                out["traj_ms"].append(tm["traj"])
                fc, ft, ch = algorithmic_work(fh, T, M, W)
                out["fma_c"] += fc
                out["fma_t"] += ft
                out["checks"] += ch
                out["free"].append(float(np.mean(fh < 0)))
        st = npp.npp_loop_read(L)
        out["waypoints_reached"] = st["waypoint"] + st["done"]
        out["n_infeasible"] = st["n_infeasible"]
        npp.npp_loop_destroy(L)
        return out

    def host_loop_pass(nsteps: int):
        """The same closed loop through the host-buffer entry point: obstacle
        copy in, plan, result copy out, synchronise, host vehicle model."""
        import ctypes
        state = sc["state"].copy()
        mission = closed_loop.Mission(sc["waypoints"], inputs.EPS)
        obs_pin = torch.empty(M, 4, dtype=torch.float32).pin_memory()
        hb = npp.npp_best()
        params_h = torch.empty(pl.n_theta, dtype=torch.float32).pin_memory()
        ctrl_h = torch.empty(T, 2, dtype=torch.float32).pin_memory()
        traj_h = torch.empty(T + 1, 4, dtype=torch.float32).pin_memory()
        warm_pin = torch.empty(pl.n_theta, dtype=torch.float32).pin_memory()
        o = npp.npp_outputs()
        o.best = ctypes.addressof(hb)
        o.params = params_h.data_ptr()
        o.controls = ctrl_h.data_ptr()
        o.trajectory = traj_h.data_ptr()
        obs = sc["obs"].copy()
        wall_ms = []
        for t in range(nsteps):
            obs_pin.copy_(torch.from_numpy(obs.astype(np.float32)))
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            npp.npp_plan_step_host(pl.h, state, mission.goal, obs_pin, M, N, T, sc["seed"], t,
                                   warm_pin if t > 0 else None, o)
            wall_ms.append((time.perf_counter() - t0) * 1e3)
            a = ctrl_h[0].numpy().astype(np.float64)
            warm_pin.copy_(params_h)
            state = closed_loop.plant_step(p, state, a)
            obs = closed_loop.advance_obstacles(obs, p["Ts"])
            mission.update(state)
        return wall_ms

    # warm-up (untimed) then K timed steps of the device path, with the SM
    # clocks sampled during them
    device_loop_pass(Wu, record=False)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    res = device_loop_pass(K, record=True)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    total_ms = float(np.sum(res["step_ms"]))
    collide_ms = float(np.sum(res["collide_ms"]))
    traj_ms = float(np.sum(res["traj_ms"]))
    e2e = None
    if not args.no_e2e:
        host_loop_pass(min(Wu, 3))
        wall = float(np.sum(host_loop_pass(K)))
        e2e = {"value": N * T * K / (wall / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": M * 16 + pl.n_theta * 4,
               "d2h_bytes_per_step": 32 + pl.n_theta * 4 + T * 8 + (T + 1) * 16}
    from paper_1904_06680_gb300 import multi
    e2e_s = N * T * K / e2e["value"] if e2e else 0.0
    total_ms, collide_ms, traj_ms, e2e_s = multi.max_over_ranks([total_ms, collide_ms, traj_ms, e2e_s], dev)
    if e2e:
        e2e["value"] = multi.whole_job_rate(N * T * K, world, e2e_s)
    value = multi.whole_job_rate(N * T * K, world, total_ms / 1e3)
    peak, peak_basis = fp32_peak(local)
    # the library's own FMA-stream microbenchmark, beside the derived peak
    fma_measured = {"ffma": npp.npp_measure_fma_peak(local, False) / 1e12,
                    "ffma2": npp.npp_measure_fma_peak(local, True) / 1e12, "unit": "T FP32-FMA/s"}
    # the library's automatic collision choice (binned from 128 points);
    # "fuse" runs the binned check inside the trajectory kernel
    cv = int(options.get("collide_variant", -1))
    binned = poly or cv == 5 or (cv < 0 and M >= 128)
    fz = int(options.get("fuse", DEFAULT_FUSE))
    fused = binned and not poly and (fz == 1 or (fz < 0 and W == 64))
    # the library's step chunks of the split binned path (option "chunks";
    # 0: two at width 64), each one trajectory and one check launch
    nch = 1
    if binned and not poly and not fused:
        nch = min(int(options.get("chunks", 0)) or (2 if W == 64 else 1), T)
    # per sampling time: plan step kernels, epilogue, vehicle and obstacle advance
    launches_per_step = (2 if fused else 1 + 2 * nch if binned and not poly else 3 if poly else 2) + 3
    # default launch shapes; the last template argument is the variant flag
    # (off: no speed limits, features in the EV frame at t)
    var = int(bool(p.get("v_limits", 0) or p.get("feature_frame", 0)))
    shape = {16: "<16,8,4,4,%d,0>" if var else "<16,8,8,3,%d,0>", 32: "<32,16,4,4,%d,0>",
             64: "<64,32,1,16,%d,8>"}[W] % var
    if fused:
        # [0] grid build, [1] the trajectory kernel with the windowed check
        fshape = {16: "<16,8,4,4,%d,0,16,4>", 32: "<32,16,4,5,%d,5,8,4>", 64: "<64,32,1,16,%d,12,8,4>"}[W] % var
        fname = "fused_kernel" + fshape
        fps = res["fma_t"] / (collide_ms / 1e3)
        rolled = res["rolled"] if res["rolled"] > 0 else float(N) * T * K
        fma_rolled = rolled * (W * W + 10 * W)
        check = {}
        if res["states"] > 0:
            # the window check's algorithmic reads (L2-resident grids): per
            # state checked the ten cell-run bounds of its query (40 B; the
            # state itself is in the warp's shared window), per candidate
            # test one point (8 B)
            wbytes = res["states"] * 40.0 + res["cand_tests"] * 8.0
            check = {"candidate_tests_per_state": res["cand_tests"] / res["states"],
                     "states_checked_per_plan_step": res["states"] / K,
                     "candidate_tests_per_s": res["cand_tests"] / (collide_ms / 1e3),
                     "bytes_per_step": wbytes / K, "achieved_gbs": wbytes / (collide_ms / 1e3) / 1e9,
                     "bytes_note": "algorithmic grid reads: 40 B per state checked (ten cell-run "
                                   "bounds), 8 B per candidate test, over the kernel's duration"}
        bin_bytes = grid_bytes(T, M)
        bin_s = traj_ms / K / 1e3
        bins = {"ms_per_step": traj_ms / K, "bytes_per_step": bin_bytes,
                "achieved_gbs": bin_bytes / bin_s / 1e9 if bin_s > 0 else None,
                "traffic": profiled_traffic("bin_build_kernel", args.workload),
                "bytes_note": "algorithmic: per grid the M points read twice (16 B), the cell-start "
                              "table and M sorted points (8 B) written; traffic = DRAM bytes per launch "
                              "from profiles/traffic.json (the grids stay in L2)"}
        roofline = {"bound": "alu", "kernel": fname, "achieved": fps / 1e12, "peak": peak / 1e12,
                    "unit": "T FP32-FMA/s", "frac": fps / peak, "traffic": profiled_traffic(fname, args.workload),
                    "peak_basis": peak_basis, "peak_measured": fma_measured,
                    "work": "MLP FMAs (W^2 + 10 W) per control step of a sample up to its first collision; "
                            "the kernel rolls a sample out to the end of the window (8 states at width 64) holding its first "
                            "collision (rolled_steps_*) and checks the window's states itself (its candidate "
                            "tests are not counted as work)",
                    "rolled_steps_per_plan_step": rolled / K,
                    "rolled_steps_of_all": rolled / (float(N) * T * K),
                    "rolled_steps_achieved": fma_rolled / (collide_ms / 1e3) / 1e12,
                    "rolled_steps_frac": fma_rolled / (collide_ms / 1e3) / peak,
                    "kernel_ms_per_step": collide_ms / K,
                    "windowed_check": check,
                    "other": {"bin_build_kernel": bins},
                    "dominant": fname}
    elif binned:
        # the binned (or polygon) check does only the candidate work of the
        # cells a state overlaps, which has no fixed algorithmic count; the
        # MLP rollout is the work every plan step must do
        tname = "traj_kernel" + shape
        cname = "bin_build_kernel + " + ("collide_poly_kernel" if poly else "collide_binned_kernel")
        fps_t = res["fma_t"] / (traj_ms / 1e3)
        coll = {"ms_per_step": collide_ms / K}
        if not poly and res["states"] > 0:
            # the check's algorithmic bytes: per state checked its stored
            # state (16 B) and the ten cell-run bounds of its query (40 B),
            # per candidate test one point (8 B), per sample its free cost
            # read and cost / first-hit written (12 B)
            nbytes = res["states"] * 56.0 + res["cand_tests"] * 8.0 + 12.0 * N * K
            coll.update(candidate_tests_per_s=res["cand_tests"] / (collide_ms / 1e3),
                        candidate_tests_per_state=res["cand_tests"] / res["states"],
                        states_per_s=res["states"] / (collide_ms / 1e3),
                        bytes_per_step=nbytes / K, achieved_gbs=nbytes / (collide_ms / 1e3) / 1e9,
                        traffic=profiled_traffic("collide_binned_kernel", args.workload),
                        bytes_note="algorithmic: 56 B per state checked (state + ten cell-run bounds), "
                                   "8 B per candidate test, 12 B per sample; traffic = DRAM bytes per "
                                   "launch from profiles/traffic.json")
        # sample-steps the trajectory launches rolled out (N T per plan step
        # in one launch; fewer in step chunks, which drop collided samples)
        rolled = res["rolled"] if res["rolled"] > 0 else float(N) * T * K
        fma_rolled = rolled * (W * W + 10 * W)
        roofline = {"bound": "alu", "kernel": tname, "achieved": fps_t / 1e12, "peak": peak / 1e12,
                    "unit": "T FP32-FMA/s", "frac": fps_t / peak, "traffic": profiled_traffic(tname, args.workload),
                    "peak_basis": peak_basis, "peak_measured": fma_measured,
                    "work": "MLP FMAs (W^2 + 10 W) per control step of a sample up to its first "
                            "collision; rolled_steps_* count every step the kernel computed",
                    "rolled_steps_per_plan_step": rolled / K,
                    "rolled_steps_of_all": rolled / (float(N) * T * K),
                    "rolled_steps_achieved": fma_rolled / (traj_ms / 1e3) / 1e12,
                    "rolled_steps_frac": fma_rolled / (traj_ms / 1e3) / peak,
                    "kernel_ms_per_step": traj_ms / K,
                    "other": {cname: coll},
                    "dominant": tname if traj_ms >= collide_ms else cname}
    else:
        tname = "traj_kernel" + shape
        cname = {0: "collide_block_kernel<16,128,1>", 1: "collide_block_kernel<8,64,2>",
                 2: "collide_warp_kernel<8,2>", 3: "collide_slice_kernel<4,2,0,2>",
                 4: "collide_slice_kernel<2,2,0,4>"}[cv if cv >= 0 else brute_auto(M, N)]
        fps_c = res["fma_c"] / (collide_ms / 1e3)
        fps_t = res["fma_t"] / (traj_ms / 1e3)
        roofline = {"bound": "alu", "kernel": cname,
                    "achieved": fps_c / 1e12, "peak": peak / 1e12, "unit": "T FP32-FMA/s",
                    "frac": fps_c / peak, "traffic": profiled_traffic(cname, args.workload),
                    "peak_basis": peak_basis, "peak_measured": fma_measured,
                    "work": "4 FMAs per point-check (two rows of the rotated inequality test) of a sample "
                            "up to its first collision",
                    "kernel_ms_per_step": collide_ms / K,
                    "point_checks_per_s": res["checks"] / (collide_ms / 1e3),
                    "other": {tname: {"ms_per_step": traj_ms / K, "achieved": fps_t / 1e12,
                                      "frac": fps_t / peak}},
                    "dominant": cname if collide_ms >= traj_ms else tname}
    # the same achieved rate against the library's measured FMA-stream peaks
    roofline["frac_of_measured"] = {k: roofline["achieved"] / fma_measured[k] for k in ("ffma", "ffma2")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wu, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc,
                       "N": N, "T": T, "M": M, "width": W, "parallelism": "replicas (rank = scene)",
                       "l2": "flushed (256 MiB write) between timed steps",
                       "timing": "sum of per-step CUDA-event durations (events captured in the "
                                 "step graph, replayed on the launching stream)"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches_per_step * K,
            "clocks": ck, "options": options,
            "free_fraction": float(np.mean(res["free"])),
            "waypoints_reached": res["waypoints_reached"], "infeasible_steps": res["n_infeasible"]}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, sc["state"], sc["waypoints"][0], sc["obs"], T,
                                            args.workload)
    pl.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def run_reference(args):
    """The CPU oracle as it stands, timed on the host cores, on the same
    closed-loop workload with a bounded number of samples per plan step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1904_06680_gb300 import closed_loop, inputs
    sc, desc = workload_setup(args.workload, args.seed)
    p = sc["preset"]
    T = sc["T"]
    M = sc["obs"].shape[0]
    cores = os.cpu_count() or 1
    Ns = 2048 if args.workload == "course" else 512
    state = sc["state"].copy()
    obs = sc["obs"].copy()
    mission = closed_loop.Mission(sc["waypoints"], inputs.EPS)
    warm = None
    times = []
    for t in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = orc.plan(p, state, mission.goal, obs, Ns, T, sc["seed"], t, warm=warm, n_threads=cores)
        dt = time.perf_counter() - t0
        if t >= args.warmup:
            times.append(dt)
        warm = r["best_theta"]
        state = closed_loop.plant_step(p, state, r["controls"][0])
        obs = closed_loop.advance_obstacles(obs, p["Ts"])
        mission.update(state)
    total = float(np.sum(times))
    value = Ns * T * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "N": sc["N"], "T": T, "M": M},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d samples per plan step (of %d) over the full horizon, "
                                       "FP64 C oracle with OpenMP" % (Ns, sc["N"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batch_cpu_baseline(bt, target_cpu_s=15.0):
    """Oracle (as it stands) on the host cores: the first scenes of the batch,
    a bounded number of samples each over their full horizon (brute-force
    checks), rollout-steps per second of wall time."""
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    done_steps, wall, used = 0.0, 0.0, 0
    for s_ in bt["scenes"]:
        if wall * cores > target_cpu_s:
            break
        o = bt["obs"][s_["obs_offset"]:s_["obs_offset"] + s_["M"]]
        st = np.asarray(s_["state"], np.float32).astype(np.float64)
        goal_ev, obs_ev = orc.frame_to_ev(st, np.asarray(s_["goal"], np.float32).astype(np.float64),
                                          np.asarray(o, np.float32).astype(np.float64))
        p = inputs_planner(s_["width"])
        K = min(s_["N"], 512)
        t0 = time.perf_counter()
        orc.rollout_samples(p, s_["seed"], 0, np.arange(K, dtype=np.int32), [0, 0, 0, st[3]], st[4:6], goal_ev,
                            obs_ev, s_["T"], n_threads=cores, record=False)
        wall += time.perf_counter() - t0
        done_steps += K * s_["T"]
        used += 1
    return {"value": done_steps / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "the first %d scenes of the batch, up to 512 samples each over the full horizon, brute-force "
                      "checks, FP64 C with OpenMP (%.1f s wall)" % (used, wall)}


def inputs_planner(width):
    from paper_1904_06680_gb300 import inputs
    return inputs.planner(width)


def run_batch(args):
    """512 reverse-parking scenes (N log-uniform 1k-64k, T 20-80, M
    log-uniform 100-20000 with 30 % moving, widths 16/32/64) planned as one
    batch of persistent launches captured in a CUDA graph; the launch shapes
    are autotuned first (untimed).  value = sum N*T / replay time."""
    import torch
    from paper_1904_06680_gb300 import autotune, inputs, npp
    rank, world, local = dist_env()
    torch.cuda.set_device(local)              # before the process group: NCCL binds the current device
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    bt = inputs.scene_batch(args.seed + rank)
    sc = bt["scenes"]
    S = len(sc)
    pl = npp.Planner(bt["preset"], max_N=1, max_T=1, max_M=1)
    B = npp.npp_batch_create(pl.h, npp.make_scenes(sc))
    off = npp.npp_batch_offsets(B, S)
    obs = torch.tensor(bt["obs"], dtype=torch.float32, device=dev)
    best = torch.zeros(S * 8, dtype=torch.int32, device=dev)
    params = torch.zeros(int(off[S, 0]), dtype=torch.float32, device=dev)
    ctrl = torch.zeros(int(off[S, 1]) * 2, dtype=torch.float32, device=dev)
    traj = torch.zeros(int(off[S, 2]) * 4, dtype=torch.float32, device=dev)
    costs = torch.zeros(int(off[S, 3]), dtype=torch.float32, device=dev)
    fh = torch.zeros(int(off[S, 3]), dtype=torch.int32, device=dev)
    out = npp.npp_batch_outputs()
    out.best, out.params, out.controls = best.data_ptr(), params.data_ptr(), ctrl.data_ptr()
    out.trajectory, out.costs, out.first_hit = traj.data_ptr(), costs.data_ptr(), fh.data_ptr()
    choice, tuned = autotune.tune_batch(B, obs, out, key="parking512", reps=1)
    npp.npp_set_timing(pl.h, True)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        npp.npp_plan_batch(B, obs, out, stream=torch.cuda.current_stream())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    K = max(1, min(args.steps, 10))
    clocks = Clocks(local)
    clocks.start()
    tot, col, trj = [], [], []
    for _ in range(K):
        flush.zero_()
        torch.cuda.synchronize()
        g.replay()
        tm = npp.npp_last_timing(pl.h)
        tot.append(tm["total"]); col.append(tm["collide"]); trj.append(tm["traj"])
    torch.cuda.synchronize()
    ck = clocks.stop()
    fhs = fh.cpu().numpy()
    steps = float(sum(s["N"] * s["T"] for s in sc))
    checks = 0.0
    for i, s in enumerate(sc):
        f = fhs[int(off[i, 3]): int(off[i, 3]) + s["N"]]
        checks += float(np.where(f < 0, s["T"] + 1, f + 1).sum()) * s["M"]
    total_ms = float(np.mean(tot))
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt[0])
    peak, peak_basis = fp32_peak(local)
    col_ms, trj_ms = float(np.mean(col)), float(np.mean(trj))
    binned = choice[0] == 1
    # MLP FMAs of live control steps, per scene width
    mlp = 0.0
    for i, s in enumerate(sc):
        f = fhs[int(off[i, 3]): int(off[i, 3]) + s["N"]]
        w = s["width"]
        mlp += float(np.where(f < 0, s["T"], f).sum()) * (w * w + 10 * w)
    fps_t = mlp / (trj_ms / 1e3)
    # per-step grids of every scene (binned check)
    bin_bytes = float(sum(grid_bytes(s["T"], s["M"]) for s in sc))
    if binned and trj_ms >= col_ms:
        # with the binned check the stage before the check holds the point
        # prologue, the grids and the trajectory kernels, the width-64 ones
        # checking their scenes window by window
        roof = {"bound": "alu", "kernel": "batch_traj_kernel (widths 16/32/64; 64 with the windowed check)",
                "achieved": fps_t / 1e12,
                "peak": peak / 1e12, "unit": "T FP32-FMA/s", "frac": fps_t / peak, "traffic": None,
                "peak_basis": peak_basis,
                "work": "MLP FMAs (W^2 + 10 W) per control step up to first collision; the time includes "
                        "the point prologue and grid build before the trajectories",
                "kernel_ms_per_step": trj_ms,
                "other": {"batch_binned_kernel (widths 16/32)": {
                    "ms_per_step": col_ms,
                    "note": "binned: checks only the points of the cells a state's disk overlaps"},
                    "obstacle_and_bin_streams": {
                        "bytes_per_step": bin_bytes,
                        "achieved_gbs_lower_bound": bin_bytes / (trj_ms / 1e3) / 1e9,
                        "note": "algorithmic bytes of the per-step grids of every scene (its M points read "
                                "twice at 16 B, the cell-start table and M sorted points at 8 B written, per "
                                "step h = 0..T); the grids are built inside the stage timed with the "
                                "trajectories, so the rate over that stage is a lower bound"}}}
    else:
        fps = 4.0 * checks / (col_ms / 1e3)
        roof = {"bound": "alu", "kernel": ("batch_binned_kernel" if binned else "batch_collide_kernel<%d>" % choice[1]),
                "achieved": fps / 1e12, "peak": peak / 1e12, "unit": "T FP32-FMA/s",
                "frac": fps / peak, "traffic": None,
                "peak_basis": peak_basis,
                "kernel_ms_per_step": col_ms, "traj_ms_per_step": trj_ms,
                "point_checks_per_s": checks / (col_ms / 1e3)}
    n_widths = len(set(s["width"] for s in sc))
    line = {"metric": METRIC, "value": world * steps / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of 512 reverse-parking scenes, N log-U[1k,64k], T U[20,80], "
                                   "M log-U[100,20000] (30% moving), widths {16,32,64}, one CUDA graph",
                       "scenes": S, "sum_N_T": steps,
                       "autotuned": {"collide": "binned" if binned else "brute force, culled tiles",
                                     "slices": choice[1], "traj_warps": choice[2]},
                       "l2": "flushed (256 MiB write) between replays"},
            "roofline": roof,
            # prologue, grids (binned), one trajectory kernel per width, check, epilogue
            "gpu_launches": (1 + (1 if binned else 0) + n_widths + 1 + 1) * K, "clocks": ck,
            "cpu_baseline": None if (args.no_cpu_baseline or rank != 0) else batch_cpu_baseline(bt),
            "free_fraction": float(np.mean(fhs < 0)),
            "infeasible_scenes": int((best.cpu().view(S, 8)[:, 1] == 2).sum())}
    npp.npp_batch_destroy(B)
    pl.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def proposal_cpu_baseline(B=256, reps=3):
    """Oracle (numpy FP64, as it stands) forward + NLL + backward + Adam step
    of the proposal network on a batch of B rows, samples per second."""
    from oracle import proposal as OP
    rng = np.random.default_rng(0)
    params = OP.init_params(0)
    X = rng.uniform(0, 1, (B, OP.N_IN))
    th = rng.standard_normal((B, OP.N_THETA))
    st = OP.adam_init()
    t0 = time.perf_counter()
    for _ in range(reps):
        c = OP.forward(params, X)
        g = OP.backward(params, c, th)
        params, st = OP.adam_step(params, g, st, 1e-4)
    wall = time.perf_counter() - t0
    return {"value": B * reps / wall, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": "%d training steps of a %d-row batch (forward with BF16 rounding, NLL, backward, Adam) "
                      "in numpy FP64 (%.1f s wall)" % (reps, B, wall)}


def run_proposal(args):
    """The learned sampling proposal on one GPU: (1) the tensor-core GEMM at
    8192^3 (roofline against the measured cuBLAS BF16 peak), (2) training
    throughput at a batch of 8192 (the network's eight GEMMs, loss, bias
    gradients, Adam), (3) a shortened training run and the plan quality of
    the mixed sampler against the plain one on held-out scenes.  value =
    training samples/s."""
    import torch
    from paper_1904_06680_gb300 import npp, proposal
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    # (1) standalone GEMM
    Mg = 8192
    g = torch.Generator(device="cpu").manual_seed(0)
    A = torch.randn(Mg, Mg, generator=g).to(torch.bfloat16).to(dev)
    Bm = torch.randn(Mg, Mg, generator=g).to(torch.bfloat16).to(dev)
    Cm = torch.empty(Mg, Mg, dtype=torch.float32, device=dev)
    for _ in range(3):
        npp.npp_gemm_bf16(A, Bm, Cm, Mg, Mg, Mg)
    torch.cuda.synchronize()
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        npp.npp_gemm_bf16(A, Bm, Cm, Mg, Mg, Mg)
    e1.record()
    torch.cuda.synchronize()
    npp.npp_gemm_status()
    gemm_ms = e0.elapsed_time(e1) / reps
    gemm_tf = 2.0 * Mg ** 3 / (gemm_ms * 1e-3) / 1e12
    del A, Bm, Cm
    # (2) training throughput
    Bt = 8192
    net = proposal.ProposalNet(batch=Bt)
    net.init(0)
    X = torch.rand(Bt, 72, device=dev)
    Th = torch.randn(Bt, 450, device=dev)
    for _ in range(args.warmup):
        net.train_step(X, Th, 1e-4)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    e0.record()
    for _ in range(args.steps):
        net.train_step(X, Th, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    step_ms = e0.elapsed_time(e1) / args.steps
    net.close()
    flops = 2.0 * Bt * (128 * 256 + 256 * 256 + 256 * 1024) + 2.0 * Bt * (1024 * 256 + 256 * 256) \
        + 2.0 * Bt * (1024 * 256 + 256 * 256 + 256 * 128)
    # (3) quality after a shortened recipe
    t0 = time.time()
    qnet, stats = proposal.train_proposal(rounds=args.rounds, S=8192, N=2048, epochs=4)
    train_s = time.time() - t0
    quality = proposal.evaluate(qnet, 0, S=192, Ns=(512, 2048, 8192, 16384), prop_frac=0.5)
    qnet.close()
    line = {"metric": "proposal training samples/s (BF16 tensor-core forward+backward+Adam)",
            "value": Bt / (step_ms * 1e-3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "learned proposal 72-256-256-900, batch 8192; quality: expert-iteration "
                                   "recipe, %d rounds of 8192 course-like scenes at N=2048, "
                                   "evaluated on 192 held-out scenes" % args.rounds,
                       "l2": "train-step working set ~100 MB (L2-resident between steps)"},
            "roofline": {"bound": "tensor", "kernel": "gemm_kernel<256> (tcgen05, M=N=K=8192)",
                         "achieved": gemm_tf, "peak": peak, "unit": "TFLOP/s", "frac": gemm_tf / peak,
                         "traffic": None, "peak_basis": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)",
                         "kernel_ms": gemm_ms,
                         "train_step_gemm_tflops": flops / (step_ms * 1e-3) / 1e12},
            "e2e": None, "gpu_launches": 14 * args.steps, "clocks": ck,
            "cpu_baseline": None if args.no_cpu_baseline else proposal_cpu_baseline(),
            "quality": {str(k): v for k, v in quality.items()},
            "training": {"rounds": args.rounds, "seconds": train_s,
                         "proposal_won_first_last": [stats[0]["proposal_won"], stats[-1]["proposal_won"]]}}
    print(json.dumps(line))


# the paper's tau_a (Step 5 of Alg. 1: 15 restarts of n = 20480 samples over
# H = 200 steps per sampling time) on its i7-7700K + Titan V, seconds, quoted
# as context: (experiment, network, obstacle points, tau_a)
PAPER_TAU = [("Exp. 2, 50 km/h, no obstacles", "NN-[5,2,2] (18 parameters)", 0, 0.036),
             ("Exp. 2", "NN-[5,10,2] (82 parameters)", 0, 0.047),
             ("Exp. 2", "NN-[5,10,10,2] (192 parameters)", 0, 0.130),
             ("Exp. 3, 4 points on a vehicle + 16 road bounds", "NN-[5,2,2]", 20, 0.090)]


def run_paper(args):
    """The paper's own Step-5 setting (Sect. V): per sampling time the hill
    climb's 15 restart rounds of n = 20480 samples over H = 200 steps, with
    the paper's vehicle and cost weights, on this library's smallest network
    (8-16-16-2, 450 parameters; the paper's have 18 to 192).  Two scenes: an
    empty road at 50 km/h (Experiment 2) and 20 points, 4 on a car ahead at
    20 km/h and 16 road bounds (Experiment 3).  value = 15 x 20480 x 200
    rollout-steps / device time per sampling time (CUDA events around each
    npp_plan_tshc call, L2 flushed between calls); the paper's tau_a on its
    Titan V is quoted beside it as context, not as a target."""
    import torch
    from paper_1904_06680_gb300 import inputs, npp
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    R = 15
    scenes = (("no obstacles (Exp. 2)", inputs.scene_paper_road(False)),
              ("20 points (Exp. 3)", inputs.scene_paper_road(True)))
    p, N, T = scenes[0][1]["preset"], scenes[0][1]["N"], scenes[0][1]["T"]
    state, goal = scenes[0][1]["state"], scenes[0][1]["goal"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    pl = npp.Planner(p, max_N=N, max_T=T, max_M=20)
    out = pl.outputs()
    rows = []
    clocks = Clocks(0)
    clocks.start()
    for label, scn in scenes:
        obs = scn["obs"]
        obs_d = torch.tensor(obs, dtype=torch.float32, device=dev)
        ms = []
        for t in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            npp.npp_plan_tshc(pl.h, state, goal, obs_d, obs.shape[0], N, T, inputs.philox_seed(0), t, None, R,
                              0.1, out)
            e1.record()
            torch.cuda.synchronize()
            if t >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        r = pl.result(N, T)
        tau = float(np.mean(ms)) / 1e3
        rows.append({"scene": label, "points": int(obs.shape[0]), "tau_s": tau,
                     "rollout_steps_per_s": R * N * T / tau, "status": r["status"],
                     "best_cost": r["best_cost"]})
    ck = clocks.stop()
    pl.close()
    tot = float(np.mean([r_["tau_s"] for r_ in rows]))
    line = {"metric": METRIC, "value": R * N * T / tot, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "the paper's Step 5: 15 restart rounds x 20480 samples x H=200 per sampling "
                                   "time, the paper's vehicle, network 8-16-16-2 (450 parameters); mean of two "
                                   "scenes (no obstacles; 20 points)",
                       "N": N, "T": T, "restarts": R, "width": 16,
                       "l2": "flushed (256 MiB write) between timed calls"},
            "scenes": rows,
            "paper_tau_s_titan_v": [{"experiment": e, "network": n, "points": m, "tau_s": t_}
                                    for e, n, m, t_ in PAPER_TAU],
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": ck}
    print(json.dumps(line))


def executed_collisions(log, obs, p):
    """Sampling times whose executed pose (log rows: x, y, phi before the
    step) has some obstacle point (at its position at that time) strictly
    inside the vehicle rectangle: an evaluation of the run, numpy."""
    bad = []
    hl, hw, co = p["half_len"], p["half_wid"], p["c_off"]
    for t in range(len(log)):
        x, y, ph = (float(v) for v in log[t, :3])
        tau = t * p["Ts"]
        dx = obs[:, 0] + tau * obs[:, 2] - x
        dy = obs[:, 1] + tau * obs[:, 3] - y
        c, s_ = np.cos(ph), np.sin(ph)
        xi, eta = c * dx + s_ * dy - co, -s_ * dx + c * dy
        if np.any((np.abs(xi) < hl) & (np.abs(eta) < hw)):
            bad.append(t)
    return bad


def run_mission(args):
    """Road missions (mission layer on the device loop: reference path,
    goal in the range field, points outside it hidden) for several scene
    seeds: outcome (completed, collision-free, sampling times needed) and the
    plan-step throughput over all sampling times (device events captured in
    each step's graph; L2 flushed between steps)."""
    import torch
    from paper_1904_06680_gb300 import inputs, npp
    rank, world, local = dist_env()
    torch.cuda.set_device(local)              # before the process group: NCCL binds the current device
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    n_missions = args.missions
    max_steps = 800
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    results, step_ms = [], []
    sc0 = inputs.scene_mission(0)
    N, T, W = sc0["N"], sc0["T"], sc0["preset"]["widths"][1]
    launches = 0
    clocks = Clocks(local)
    t_wall = time.perf_counter()
    clocks.start()
    for k in range(n_missions):
        sc = inputs.scene_mission(args.seed + k + rank * 1000)
        M = sc["obs"].shape[0]
        pl = npp.Planner(sc["preset"], max_N=N, max_T=T, max_M=M, device=local)
        obs = torch.tensor(sc["obs"], dtype=torch.float32, device=dev)
        L = npp.npp_loop_create_mission(pl.h, sc["state"], sc["ref"], sc["field"], sc["window"], 1, inputs.EPS,
                                        obs, M, N, T, sc["seed"], max_log=max_steps)
        done_at = None
        for t in range(max_steps):
            flush.zero_()
            torch.cuda.synchronize()
            npp.npp_loop_run(L, 1)
            tm = npp.npp_loop_last_timing(L)
            if t >= args.warmup or k > 0:
                step_ms.append(tm["total"])
            # trajectories, collision check (+ grid build when binned), epilogue, vehicle, points
            launches += 6 if M >= 128 else 5
            st = npp.npp_loop_read(L)
            if st["done"]:
                done_at = st["t"]
                break
        st = npp.npp_loop_read(L)
        log = npp.npp_loop_log(L, max_steps)
        npp.npp_loop_destroy(L)
        pl.close()
        hits = executed_collisions(log, sc["obs"], sc["preset"])
        results.append(dict(seed=args.seed + k, completed=bool(st["done"]), steps=int(st["t"]),
                            done_at=done_at, collisions=len(hits), n_infeasible=int(st["n_infeasible"])))
    # the reverse parking mission (Experiment 5) over the same seeds: outcome only
    parking = []
    for k in range(n_missions):
        sp = inputs.scene_parking(args.seed + k + rank * 1000)
        Mp = sp["obs"].shape[0]
        pl = npp.Planner(sp["preset"], max_N=sp["N"], max_T=sp["T"], max_M=Mp, device=local)
        # the hill climb of Sect. II-D in every sampling time (4 rounds)
        npp.npp_set_loop_restarts(pl.h, 4, 0.1)
        obs = torch.tensor(sp["obs"], dtype=torch.float32, device=dev)
        L = npp.npp_loop_create(pl.h, sp["state"], sp["waypoints"], inputs.EPS, obs, Mp, sp["N"], sp["T"],
                                sp["seed"], max_log=max_steps)
        for t in range(max_steps):
            npp.npp_loop_run(L, 1)
            st = npp.npp_loop_read(L)
            if st["done"]:
                break
        log = npp.npp_loop_log(L, max_steps)
        npp.npp_loop_destroy(L)
        pl.close()
        parking.append(dict(seed=args.seed + k, completed=bool(st["done"]), steps=int(st["t"]),
                            collisions=len(executed_collisions(log, sp["obs"], sp["preset"]))))
    ck = clocks.stop()
    wall = time.perf_counter() - t_wall
    tot_ms = float(np.sum(step_ms))
    units = float(N * T * len(step_ms))
    if world > 1:
        # every rank flies its own missions (seeds offset by rank): units of
        # all ranks over the slowest rank's device time
        import torch.distributed as dist
        from paper_1904_06680_gb300 import multi
        u = torch.tensor([units], dtype=torch.float64, device=dev)
        dist.all_reduce(u)
        units = float(u.item())
        tot_ms = multi.max_over_ranks([tot_ms], dev)[0]
        dist.barrier()
        dist.destroy_process_group()
    ok = [r for r in results if r["completed"] and r["collisions"] == 0]
    line = {"metric": "rollout_steps_per_s", "value": units / (tot_ms * 1e-3),
            "unit": "rollout-steps/s", "n_gpus": world, "steps": len(step_ms), "warmup": args.warmup,
            "ms_per_step": tot_ms / len(step_ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mission", "parallelism": "replicas (rank = mission seeds)", "description":
                       "road missions (reference path along a winding two-lane road, 150 m; six parked cars "
                       "in the lane, an oncoming car; range field 25/8/10 m with points outside it hidden): "
                       "N=%d samples, T=%d, MLP 8-%d-%d-2, one plan step per sampling time" % (N, T, W, W),
                       "missions": n_missions, "l2": "flushed (256 MiB write) between sampling times"},
            "mission": {"completed": sum(r["completed"] for r in results), "collision_free_and_completed": len(ok),
                        "of": len(results),
                        "sampling_times_mean": float(np.mean([r["steps"] for r in ok])) if ok else None,
                        "sampling_times_max": max((r["steps"] for r in ok), default=None),
                        "runs": results, "wall_s": wall},
            "parking": {"completed": sum(r["completed"] for r in parking),
                        "collision_free_and_completed": sum(r["completed"] and r["collisions"] == 0 for r in parking),
                        "of": len(parking), "description": "reverse parking (Experiment 5: auxiliary waypoint, "
                        "then the slot), N=16384, T=60, MLP 8-16-16-2, 4 hill-climb rounds per sampling time "
                        "(sigma_pert 0.1)", "runs": parking},
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": ck}
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        if args.workload in ("batch", "proposal", "mission", "paper"):
            args.workload = "course"
        run_reference(args)
    elif args.workload == "mission":
        run_mission(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "proposal":
        run_proposal(args)
    elif args.workload == "paper":
        run_paper(args)
    else:
        run_npp(args)


if __name__ == "__main__":
    main()
