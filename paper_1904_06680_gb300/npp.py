"""Thin ctypes binding of libnpp.so (the C ABI in include/npp.h).

The functions keep the C names and only marshal arguments: torch tensors
provide device memory and streams, every step of the planner runs in the
library's CUDA kernels.  The first call into the library raises if it has not
been built (there is no CPU fallback).
"""
import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnpp.so")

NPP_OK, NPP_INVALID_ARG, NPP_INFEASIBLE, NPP_CUDA_ERROR, NPP_DEVICE_TIMEOUT, NPP_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "INFEASIBLE", 3: "CUDA_ERROR", 4: "DEVICE_TIMEOUT",
                5: "UNSUPPORTED"}


class NppError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("npp status %s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class npp_config(C.Structure):
    _fields_ = [(n, C.c_float) for n in (
        "lf", "lr", "delta_max", "delta_rate_max", "u_min", "u_max", "Ts",
        "half_len", "half_wid", "c_off", "dxi_n", "deta_n", "dphi_n", "dv_n",
        "w_pos", "w_phi", "w_v", "w_effort")] + [
        ("n_in", C.c_int32), ("width", C.c_int32), ("max_N", C.c_int32),
        ("max_T", C.c_int32), ("max_M", C.c_int32),
        ("feature_frame", C.c_int32), ("v_limits", C.c_int32), ("v_min", C.c_float), ("v_max", C.c_float)]


class npp_state(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("x", "y", "phi", "v", "a_prev0", "a_prev1")]


class npp_goal(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("x", "y", "phi", "v")]


class npp_best(C.Structure):
    _fields_ = [("best_idx", C.c_int32), ("status", C.c_int32), ("best_cost", C.c_float),
                ("first_hit", C.c_int32), ("reserved", C.c_int32 * 4)]


class npp_loop_state(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("x", "y", "phi", "v", "a_prev0", "a_prev1")] + [
        (n, C.c_int32) for n in ("t", "waypoint", "done", "status", "best_idx", "n_infeasible")] + [
        ("best_cost", C.c_float), ("space_index", C.c_int32), ("stop", C.c_int32), ("reserved", C.c_int32)]


class npp_scene(C.Structure):
    _fields_ = [("state", npp_state), ("goal", npp_goal), ("N", C.c_int32), ("T", C.c_int32),
                ("M", C.c_int32), ("width", C.c_int32), ("obs_offset", C.c_int64),
                ("seed", C.c_uint64), ("t_index", C.c_uint32), ("reserved", C.c_int32)]


class npp_batch_outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("best", "params", "controls", "trajectory", "costs",
                                          "first_hit")]


class npp_proposal_config(C.Structure):
    _fields_ = [("batch", C.c_int32), ("ls_min", C.c_float), ("ls_max", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("device", C.c_int32)]


class npp_outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("best", "params", "controls", "trajectory", "costs",
                                          "first_hit", "sample_traj", "sample_ctrl")]


EXPORTS = ("npp_create", "npp_destroy", "npp_last_error", "npp_n_theta", "npp_plan_step", "npp_set_footprint",
           "npp_plan_step_host", "npp_rollout_params", "npp_sample_params", "npp_set_timing",
           "npp_last_timing", "npp_set_option", "npp_plan_step_noalloc", "npp_loop_create",
           "npp_loop_run", "npp_loop_read", "npp_loop_log", "npp_loop_destroy", "npp_loop_samples",
           "npp_loop_last_timing", "npp_batch_create", "npp_batch_update", "npp_batch_offsets",
           "npp_plan_batch", "npp_batch_destroy", "npp_batch_set_option", "npp_math_eval",
           "npp_proposal_create", "npp_proposal_destroy", "npp_proposal_n_params",
           "npp_proposal_set_params", "npp_proposal_get_params", "npp_proposal_get_grads",
           "npp_proposal_encode", "npp_proposal_forward", "npp_proposal_train_step",
           "npp_plan_step_proposal", "npp_gemm_bf16", "npp_gemm_status", "npp_plan_tshc",
           "npp_loop_create_mission", "npp_loop_points", "npp_measure_fma_peak", "npp_set_loop_restarts", "npp_last_counts",
           "npp_wait_probe", "npp_inject_fault")

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnpp.so is not built: run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        P, I32, U32, U64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64
        L.npp_create.argtypes = [C.POINTER(P), C.POINTER(npp_config), I32]
        L.npp_destroy.argtypes = [P]
        L.npp_last_error.argtypes = [P]
        L.npp_last_error.restype = C.c_char_p
        L.npp_n_theta.argtypes = [C.POINTER(npp_config)]
        L.npp_n_theta.restype = I32
        L.npp_proposal_n_params.restype = I32
        L.npp_plan_step.argtypes = [P, C.POINTER(npp_state), C.POINTER(npp_goal), P, I32, I32, I32,
                                    U64, U32, P, C.POINTER(npp_outputs), P]
        L.npp_plan_step_host.argtypes = [P, C.POINTER(npp_state), C.POINTER(npp_goal), P, I32, I32,
                                         I32, U64, U32, P, C.POINTER(npp_outputs)]
        L.npp_rollout_params.argtypes = [P, C.POINTER(npp_state), C.POINTER(npp_goal), P, I32, P, I32,
                                         I32, P, P, P, P, P]
        L.npp_sample_params.argtypes = [U64, U32, U32, I32, I32, I32, P, P]
        L.npp_set_timing.argtypes = [P, I32]
        L.npp_set_option.argtypes = [P, C.c_char_p, I32]
        L.npp_set_footprint.argtypes = [P, C.c_void_p, C.c_void_p, I32]
        L.npp_measure_fma_peak.argtypes = [I32, I32, C.POINTER(C.c_double)]
        L.npp_wait_probe.argtypes = [C.c_int64, I32, C.POINTER(I32)]
        L.npp_inject_fault.argtypes = [P]
        L.npp_loop_create.argtypes = [P, C.POINTER(npp_state), P, I32, P, P, I32, I32, I32, U64, I32,
                                      C.POINTER(P)]
        L.npp_loop_run.argtypes = [P, I32, P]
        L.npp_set_loop_restarts.argtypes = [P, I32, C.c_float]
        L.npp_last_counts.argtypes = [P, C.POINTER(C.c_uint64), I32]
        L.npp_loop_read.argtypes = [P, C.POINTER(npp_loop_state)]
        L.npp_loop_log.argtypes = [P, P, I32, C.POINTER(I32)]
        L.npp_loop_destroy.argtypes = [P]
        L.npp_loop_samples.argtypes = [P, P, P]
        L.npp_loop_last_timing.argtypes = [P, C.POINTER(C.c_float), I32]
        L.npp_batch_create.argtypes = [P, P, I32, C.POINTER(P)]
        L.npp_batch_update.argtypes = [P, P]
        L.npp_batch_offsets.argtypes = [P, P]
        L.npp_plan_batch.argtypes = [P, P, C.POINTER(npp_batch_outputs), P]
        L.npp_batch_destroy.argtypes = [P]
        L.npp_batch_set_option.argtypes = [P, C.c_char_p, I32]
        L.npp_plan_step_noalloc.argtypes = [C.POINTER(npp_config), C.POINTER(npp_state),
                                            C.POINTER(npp_goal), P, I32, I32, I32, U64, U32, P,
                                            C.POINTER(npp_outputs), P]
        L.npp_last_timing.argtypes = [P, C.POINTER(C.c_float), I32]
        L.npp_math_eval.argtypes = [I32, P, I32, P, P, P]
        L.npp_proposal_create.argtypes = [C.POINTER(npp_proposal_config), C.POINTER(P)]
        L.npp_proposal_destroy.argtypes = [P]
        L.npp_proposal_n_params.argtypes = []
        L.npp_proposal_set_params.argtypes = [P, P]
        L.npp_proposal_get_params.argtypes = [P, P]
        L.npp_proposal_get_grads.argtypes = [P, P]
        L.npp_proposal_encode.argtypes = [P, P, I32, P, P, P]
        L.npp_proposal_forward.argtypes = [P, P, I32, P, P, P]
        L.npp_proposal_train_step.argtypes = [P, P, P, C.c_float, P, P]
        L.npp_plan_step_proposal.argtypes = [P, C.POINTER(npp_state), C.POINTER(npp_goal), P, I32, I32,
                                             I32, U64, U32, P, P, P, I32, C.POINTER(npp_outputs), P]
        L.npp_gemm_bf16.argtypes = [P, P, P, I32, I32, I32, P]
        L.npp_plan_tshc.argtypes = [P, C.POINTER(npp_state), C.POINTER(npp_goal), P, I32, I32, I32, U64, U32, P,
                                    I32, C.c_float, C.POINTER(npp_outputs), P]
        L.npp_gemm_status.argtypes = []
        for name in EXPORTS:
            if name not in ("npp_last_error", "npp_n_theta", "npp_proposal_n_params"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


# ------------------------------------------------------------------ helpers
def make_config(p: dict, max_N: int, max_T: int, max_M: int) -> npp_config:
    c = npp_config()
    for name, _ in npp_config._fields_[:18]:
        setattr(c, name, float(p[name]))
    widths = tuple(p["widths"])
    c.n_in = widths[0]
    c.width = widths[1]
    c.max_N, c.max_T, c.max_M = int(max_N), int(max_T), int(max_M)
    c.feature_frame = int(p.get("feature_frame", 0))
    c.v_limits = int(p.get("v_limits", 0))
    c.v_min = float(p.get("v_min", 0.0))
    c.v_max = float(p.get("v_max", 0.0))
    return c


def make_state(s) -> npp_state:
    return npp_state(*[float(v) for v in s])


def make_goal(g) -> npp_goal:
    return npp_goal(*[float(v) for v in g])


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(status, handle=None):
    if status not in (NPP_OK, NPP_INFEASIBLE):
        raise NppError(status, npp_last_error(handle))
    return status


# ------------------------------------------------------------------ C names
def npp_create(cfg: npp_config, device: int = 0):
    h = C.c_void_p()
    _check(lib().npp_create(C.byref(h), C.byref(cfg), int(device)))
    return h


def npp_destroy(h):
    return lib().npp_destroy(h)


def npp_last_error(h=None) -> str:
    r = lib().npp_last_error(h)
    return r.decode() if r else ""


def npp_measure_fma_peak(device=0, packed=False):
    """FP32 FMAs per second on independent FMA streams (scalar or packed)."""
    v = C.c_double()
    _check(lib().npp_measure_fma_peak(int(device), int(bool(packed)), C.byref(v)))
    return v.value


def npp_set_footprint(h, pieces):
    """General footprint: a list of convex pieces, each an array of
    counter-clockwise (x, y) vertices in the vehicle's frame; [] or None
    restores the rectangle."""
    import numpy as np
    pieces = [np.asarray(q, np.float32).reshape(-1, 2) for q in (pieces or [])]
    if not pieces:
        return _check(lib().npp_set_footprint(h, None, None, 0), h)
    start = np.ascontiguousarray(np.cumsum([0] + [len(q) for q in pieces]), np.int32)
    verts = np.ascontiguousarray(np.concatenate(pieces), np.float32)
    return _check(lib().npp_set_footprint(h, verts.ctypes.data_as(C.c_void_p), start.ctypes.data_as(C.c_void_p),
                                          len(pieces)), h)


def npp_n_theta(cfg: npp_config) -> int:
    return lib().npp_n_theta(C.byref(cfg))


def npp_plan_step(h, state, goal, obs, M, N, T, seed, t_index, warm, out: npp_outputs, stream=None):
    """obs / warm: CUDA tensors (or None); out: npp_outputs of device pointers."""
    return _check(lib().npp_plan_step(h, C.byref(make_state(state)), C.byref(make_goal(goal)),
                                      _ptr(obs), int(M), int(N), int(T), int(seed), int(t_index),
                                      _ptr(warm), C.byref(out), _stream(stream)), h)


def npp_plan_step_noalloc(cfg: npp_config, state, goal, obs, M, N, T, seed, t_index, warm,
                          out: npp_outputs, stream=None):
    """Plan step that allocates no device memory (fixed static workspace);
    for callers that cannot call cudaMalloc.  obs / warm: CUDA tensors or
    None; out: npp_outputs of device pointers."""
    return _check(lib().npp_plan_step_noalloc(C.byref(cfg), C.byref(make_state(state)),
                                              C.byref(make_goal(goal)), _ptr(obs), int(M), int(N),
                                              int(T), int(seed), int(t_index), _ptr(warm),
                                              C.byref(out), _stream(stream)))


def npp_plan_step_host(h, state, goal, obs, M, N, T, seed, t_index, warm, out: npp_outputs):
    """obs / warm: host (CPU) tensors; out: npp_outputs of host pointers."""
    return _check(lib().npp_plan_step_host(h, C.byref(make_state(state)), C.byref(make_goal(goal)),
                                           _ptr(obs), int(M), int(N), int(T), int(seed),
                                           int(t_index), _ptr(warm), C.byref(out)), h)


def npp_rollout_params(h, state, goal, obs, M, theta, K, T, costs, first_hit, sample_traj=None,
                       sample_ctrl=None, stream=None):
    return _check(lib().npp_rollout_params(h, C.byref(make_state(state)), C.byref(make_goal(goal)),
                                           _ptr(obs), int(M), _ptr(theta), int(K), int(T),
                                           _ptr(costs), _ptr(first_hit), _ptr(sample_traj),
                                           _ptr(sample_ctrl), _stream(stream)), h)


def npp_sample_params(seed, t_index, stream_id, n0, K, n_theta, out, stream=None):
    return _check(lib().npp_sample_params(int(seed), int(t_index), int(stream_id), int(n0), int(K),
                                          int(n_theta), _ptr(out), _stream(stream)))


def npp_math_eval(fn, x, y, y2=None, stream=None):
    """fn 0 tanh, 1 tan, 2 sin/cos (y, y2) of the rollout on CUDA tensors."""
    return _check(lib().npp_math_eval(int(fn), _ptr(x), int(x.numel()), _ptr(y), _ptr(y2),
                                      _stream(stream)))


# ------------------------------------------------------------------ proposal
def npp_proposal_create(batch, ls_min=-3.0, ls_max=1.0, beta1=0.9, beta2=0.999, eps=1e-8, device=0):
    cfg = npp_proposal_config(int(batch), ls_min, ls_max, beta1, beta2, eps, int(device))
    P = C.c_void_p()
    _check(lib().npp_proposal_create(C.byref(cfg), C.byref(P)))
    return P


def npp_proposal_destroy(P):
    return lib().npp_proposal_destroy(P)


def npp_proposal_n_params():
    return int(lib().npp_proposal_n_params())


def npp_proposal_set_params(P, vec):
    import numpy as np
    v = np.ascontiguousarray(vec, dtype=np.float32)
    assert v.size == npp_proposal_n_params()
    return _check(lib().npp_proposal_set_params(P, v.ctypes.data_as(C.c_void_p)))


def npp_proposal_get_params(P):
    import numpy as np
    v = np.zeros(npp_proposal_n_params(), np.float32)
    _check(lib().npp_proposal_get_params(P, v.ctypes.data_as(C.c_void_p)))
    return v


def npp_proposal_get_grads(P):
    import numpy as np
    v = np.zeros(npp_proposal_n_params(), np.float32)
    _check(lib().npp_proposal_get_grads(P, v.ctypes.data_as(C.c_void_p)))
    return v


def npp_proposal_encode(h, scenes_dev, S, obs, x, stream=None):
    """scenes_dev: CUDA uint8 tensor holding S npp_scene records."""
    return _check(lib().npp_proposal_encode(h, _ptr(scenes_dev), int(S), _ptr(obs), _ptr(x),
                                            _stream(stream)))


def npp_proposal_forward(P, x, n, mean, std, stream=None):
    return _check(lib().npp_proposal_forward(P, _ptr(x), int(n), _ptr(mean), _ptr(std), _stream(stream)))


def npp_proposal_train_step(P, x, theta, lr, loss=None, stream=None):
    return _check(lib().npp_proposal_train_step(P, _ptr(x), _ptr(theta), float(lr), _ptr(loss),
                                                _stream(stream)))


def npp_plan_step_proposal(h, state, goal, obs, M, N, T, seed, t_index, warm, mean, std, N_prop,
                           out: "npp_outputs", stream=None):
    return _check(lib().npp_plan_step_proposal(h, C.byref(make_state(state)), C.byref(make_goal(goal)),
                                               _ptr(obs), int(M), int(N), int(T), int(seed), int(t_index),
                                               _ptr(warm), _ptr(mean), _ptr(std), int(N_prop),
                                               C.byref(out), _stream(stream)), h)


def npp_plan_tshc(h, state, goal, obs, M, N, T, seed, t_index, warm, n_restarts, sigma_pert,
                  out: "npp_outputs", stream=None):
    return _check(lib().npp_plan_tshc(h, C.byref(make_state(state)), C.byref(make_goal(goal)), _ptr(obs), int(M),
                                      int(N), int(T), int(seed), int(t_index), _ptr(warm), int(n_restarts),
                                      float(sigma_pert), C.byref(out), _stream(stream)), h)


def npp_gemm_bf16(A, B, Cout, M, N, K, stream=None):
    """A [M][K], B [N][K] CUDA bfloat16 tensors; Cout [M][N] float32."""
    return _check(lib().npp_gemm_bf16(_ptr(A), _ptr(B), _ptr(Cout), int(M), int(N), int(K),
                                      _stream(stream)))


def npp_gemm_status():
    return _check(lib().npp_gemm_status())


def scenes_to_device(scenes_ctypes, device=0):
    """Copy a ctypes npp_scene array to a CUDA uint8 tensor."""
    raw = bytes(scenes_ctypes)
    t = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(torch.device("cuda", device))
    return t


def npp_set_option(h, name: str, value: int):
    return _check(lib().npp_set_option(h, name.encode(), int(value)), h)


def npp_set_timing(h, enable: bool):
    return _check(lib().npp_set_timing(h, 1 if enable else 0), h)


def npp_last_timing(h):
    """Stage times of the last timed call in ms: dict with keys traj,
    collide, epilogue, total."""
    t = (C.c_float * 4)()
    _check(lib().npp_last_timing(h, t, 4), h)
    return dict(traj=t[0], collide=t[1], epilogue=t[2], total=t[3])


def npp_loop_create(h, state, waypoints, eps, obs, M, N, T, seed, max_log=1024):
    """waypoints: array-like [n_wp][4]; eps: 4 tolerances; obs: CUDA tensor."""
    import numpy as np
    wp = np.ascontiguousarray(waypoints, dtype=np.float32).reshape(-1, 4)
    ep = np.ascontiguousarray(eps, dtype=np.float32).reshape(4)
    L = C.c_void_p()
    _check(lib().npp_loop_create(h, C.byref(make_state(state)), wp.ctypes.data_as(C.c_void_p),
                                 wp.shape[0], ep.ctypes.data_as(C.c_void_p), _ptr(obs), int(M),
                                 int(N), int(T), int(seed), int(max_log), C.byref(L)), h)
    return L


class npp_mission(C.Structure):
    _fields_ = [("range_front", C.c_float), ("range_back", C.c_float), ("range_side", C.c_float),
                ("window", C.c_int32), ("hide_outside", C.c_int32)]


def npp_loop_create_mission(h, state, ref, field, window, hide_outside, eps, obs, M, N, T, seed, max_log=1024):
    """ref: array-like [n_ref][4] reference setpoints; field: (front, back,
    side) of the range field; obs: CUDA tensor or None."""
    import numpy as np
    rp = np.ascontiguousarray(ref, dtype=np.float32).reshape(-1, 4)
    ep = np.ascontiguousarray(eps, dtype=np.float32).reshape(4)
    m = npp_mission(float(field[0]), float(field[1]), float(field[2]), int(window), int(hide_outside))
    L = C.c_void_p()
    _check(lib().npp_loop_create_mission(h, C.byref(make_state(state)), rp.ctypes.data_as(C.c_void_p),
                                         rp.shape[0], C.byref(m), ep.ctypes.data_as(C.c_void_p), _ptr(obs),
                                         int(M), int(N), int(T), int(seed), int(max_log), C.byref(L)), h)
    return L


def npp_last_counts(h):
    """(candidate point tests, states checked, sample-steps rolled out) of
    the last timed plan step with the binned collision check (synchronises)."""
    c = (C.c_uint64 * 3)()
    _check(lib().npp_last_counts(h, c, 3), h)
    return int(c[0]), int(c[1]), int(c[2])


def npp_wait_probe(limit_cycles: int, arrive: bool):
    """Run the library's bounded mbarrier wait on a barrier whose one arrival
    happens (arrive) or never does; True if the wait saw it complete."""
    v = C.c_int32(-1)
    _check(lib().npp_wait_probe(int(limit_cycles), int(bool(arrive)), C.byref(v)))
    return v.value == 1


def npp_inject_fault(h):
    """Set the handle's device fault flag as a timed-out wait would."""
    _check(lib().npp_inject_fault(h), h)


def npp_set_loop_restarts(h, n_restarts: int, sigma_pert: float = 0.0):
    """Hill-climb rounds per sampling time of loops created afterwards on h
    (1: the plan step alone)."""
    return _check(lib().npp_set_loop_restarts(h, int(n_restarts), float(sigma_pert)), h)


def npp_loop_points(L, M):
    """The M points (world frame, x, y, vx, vy) the next plan step sees."""
    import numpy as np
    out = np.zeros((max(M, 1), 4), np.float32)
    _check(lib().npp_loop_points(L, out.ctypes.data_as(C.c_void_p)))
    return out[:M]


def npp_loop_run(L, steps, stream=None):
    return _check(lib().npp_loop_run(L, int(steps), _stream(stream)))


def npp_loop_read(L) -> dict:
    st = npp_loop_state()
    _check(lib().npp_loop_read(L, C.byref(st)))
    return {n: getattr(st, n) for n, _ in npp_loop_state._fields_ if n != "reserved"}


def npp_loop_log(L, max_rows=1024):
    import numpy as np
    out = np.zeros((max_rows, 8), np.float32)
    rows = C.c_int32()
    _check(lib().npp_loop_log(L, out.ctypes.data_as(C.c_void_p), int(max_rows), C.byref(rows)))
    return out[: rows.value]


def npp_loop_destroy(L):
    return lib().npp_loop_destroy(L)


def npp_loop_samples(L, N):
    """(costs[N], first_hit[N]) of the last replayed step (numpy, synchronous)."""
    import numpy as np
    costs = np.zeros(N, np.float32)
    fh = np.zeros(N, np.int32)
    _check(lib().npp_loop_samples(L, costs.ctypes.data_as(C.c_void_p), fh.ctypes.data_as(C.c_void_p)))
    return costs, fh


def npp_loop_last_timing(L):
    t = (C.c_float * 4)()
    _check(lib().npp_loop_last_timing(L, t, 4))
    return dict(traj=t[0], collide=t[1], epilogue=t[2], total=t[3])


def make_scenes(descs):
    """descs: list of dicts with state, goal, N, T, M, width, obs_offset, seed,
    t_index -> ctypes array of npp_scene."""
    arr = (npp_scene * len(descs))()
    for i, d in enumerate(descs):
        arr[i].state = make_state(d["state"])
        arr[i].goal = make_goal(d["goal"])
        arr[i].N, arr[i].T, arr[i].M, arr[i].width = int(d["N"]), int(d["T"]), int(d["M"]), int(d["width"])
        arr[i].obs_offset = int(d["obs_offset"])
        arr[i].seed = int(d["seed"])
        arr[i].t_index = int(d.get("t_index", 0))
    return arr


def npp_batch_create(h, scenes):
    B = C.c_void_p()
    _check(lib().npp_batch_create(h, C.cast(scenes, C.c_void_p), len(scenes), C.byref(B)), h)
    return B


def npp_batch_update(B, scenes):
    return _check(lib().npp_batch_update(B, C.cast(scenes, C.c_void_p)))


def npp_batch_offsets(B, S):
    import numpy as np
    off = np.zeros((S + 1, 4), np.int64)
    _check(lib().npp_batch_offsets(B, off.ctypes.data_as(C.c_void_p)))
    return off


def npp_plan_batch(B, obs, out: npp_batch_outputs, stream=None):
    return _check(lib().npp_plan_batch(B, _ptr(obs), C.byref(out), _stream(stream)))


def npp_batch_destroy(B):
    return lib().npp_batch_destroy(B)


def npp_batch_set_option(B, name: str, value: int):
    return _check(lib().npp_batch_set_option(B, name.encode(), int(value)))


# ------------------------------------------------------------------ convenience
class Planner:
    """Owns a handle and the output tensors of one plan step on one device."""

    def __init__(self, preset: dict, max_N: int, max_T: int, max_M: int, device: int = 0,
                 record_samples: bool = False):
        self.cfg = make_config(preset, max_N, max_T, max_M)
        self.device = torch.device("cuda", device)
        self.h = npp_create(self.cfg, device)
        if preset.get("footprint"):
            npp_set_footprint(self.h, preset["footprint"])
        self.n_theta = npp_n_theta(self.cfg)
        d = self.device
        self.best = torch.zeros(8, dtype=torch.int32, device=d)
        self.params = torch.zeros(self.n_theta, dtype=torch.float32, device=d)
        self.controls = torch.zeros(max_T, 2, dtype=torch.float32, device=d)
        self.trajectory = torch.zeros(max_T + 1, 4, dtype=torch.float32, device=d)
        self.costs = torch.zeros(max_N, dtype=torch.float32, device=d)
        self.first_hit = torch.zeros(max_N, dtype=torch.int32, device=d)
        self.record_samples = record_samples
        self.max_N, self.max_T = max_N, max_T
        if record_samples:
            self.sample_traj = torch.zeros((max_T + 1) * max_N * 4, dtype=torch.float32, device=d)
            self.sample_ctrl = torch.zeros(max_T * max_N * 2, dtype=torch.float32, device=d)

    def outputs(self) -> npp_outputs:
        o = npp_outputs()
        o.best = self.best.data_ptr()
        o.params = self.params.data_ptr()
        o.controls = self.controls.data_ptr()
        o.trajectory = self.trajectory.data_ptr()
        o.costs = self.costs.data_ptr()
        o.first_hit = self.first_hit.data_ptr()
        if self.record_samples:
            o.sample_traj = self.sample_traj.data_ptr()
            o.sample_ctrl = self.sample_ctrl.data_ptr()
        return o

    def plan(self, state, goal, obs, N, T, seed, t_index=0, warm=None, stream=None):
        """Queue one plan step; obs is a CUDA float32 tensor [M, 4]."""
        M = 0 if obs is None else obs.shape[0]
        npp_plan_step(self.h, state, goal, obs, M, N, T, seed, t_index, warm, self.outputs(), stream)

    def result(self, N, T):
        """Host copies of the last plan step's outputs (synchronises)."""
        b = self.best.cpu()
        best_cost = b[2:3].view(torch.float32).item()
        r = dict(best_idx=int(b[0]), status=int(b[1]), best_cost=best_cost, first_hit_best=int(b[3]),
                 params=self.params.cpu().numpy(), controls=self.controls[:T].cpu().numpy(),
                 trajectory=self.trajectory[:T + 1].cpu().numpy(), costs=self.costs[:N].cpu().numpy(),
                 first_hit=self.first_hit[:N].cpu().numpy())
        if self.record_samples:
            r["sample_traj"] = self.sample_traj[:(T + 1) * N * 4].view(T + 1, N, 4).cpu().numpy()
            r["sample_ctrl"] = self.sample_ctrl[:T * N * 2].view(T, N, 2).cpu().numpy()
        return r

    def close(self):
        if self.h is not None:
            npp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
