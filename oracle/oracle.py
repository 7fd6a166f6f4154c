"""ctypes wrapper around the FP64 CPU oracle (oracle/npp_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  It takes a plain configuration dict (the
presets live in the seeded-input module) and numpy arrays; it imports nothing
from the CUDA package.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

MAX_LAYERS = 8


class OrcConfig(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "lf", "lr", "delta_max", "delta_rate_max", "u_min", "u_max", "Ts",
        "half_len", "half_wid", "c_off", "dxi_n", "deta_n", "dphi_n", "dv_n",
        "w_pos", "w_phi", "w_v", "w_effort")] + [
        ("n_layers", C.c_int32), ("widths", C.c_int32 * (MAX_LAYERS + 1)),
        ("feature_frame", C.c_int32), ("v_limits", C.c_int32), ("v_min", C.c_double), ("v_max", C.c_double),
        ("fp_pieces", C.c_int32), ("fp_start", C.POINTER(C.c_int32)), ("fp_verts", C.POINTER(C.c_double))]

N_FLOAT = 18


def make_config(p: dict) -> OrcConfig:
    """Preset dict -> FP64 config; the variant keys (feature_frame, v_limits,
    v_min, v_max, footprint) are optional and default to off.  footprint: a
    list of convex pieces, each an array of counter-clockwise vertices (x, y)
    in the vehicle's frame."""
    c = OrcConfig()
    for name, _ in OrcConfig._fields_[:N_FLOAT]:
        setattr(c, name, float(p[name]))
    widths = list(p["widths"])
    c.n_layers = len(widths) - 1
    for i, w in enumerate(widths):
        c.widths[i] = int(w)
    c.feature_frame = int(p.get("feature_frame", 0))
    c.v_limits = int(p.get("v_limits", 0))
    c.v_min = float(p.get("v_min", 0.0))
    c.v_max = float(p.get("v_max", 0.0))
    fp = p.get("footprint")
    if fp:
        pieces = [np.asarray(q, np.float64).reshape(-1, 2) for q in fp]
        start = np.ascontiguousarray(np.cumsum([0] + [len(q) for q in pieces]), np.int32)
        verts = np.ascontiguousarray(np.concatenate(pieces))
        c._keep = (start, verts)                  # alive as long as the config
        c.fp_pieces = len(pieces)
        c.fp_start = start.ctypes.data_as(C.POINTER(C.c_int32))
        c.fp_verts = verts.ctypes.data_as(C.POINTER(C.c_double))
    return c


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_P = C.POINTER(OrcConfig)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_n_theta.argtypes = [_P]
        L.orc_n_theta.restype = C.c_int
        L.orc_philox.argtypes = [_U, _U, _U]
        L.orc_u24.argtypes = [C.c_uint32]
        L.orc_u24.restype = C.c_float
        L.orc_ln32.argtypes = [C.c_float]
        L.orc_ln32.restype = C.c_float
        L.orc_sincos2pi32.argtypes = [C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.orc_normal_pair.argtypes = [C.c_uint32, C.c_uint32, _F]
        L.orc_theta.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, _F]
        L.orc_frame_to_ev.argtypes = [_D, _D, _D, C.c_int, _D, _D]
        L.orc_features.argtypes = [_P, _D, _D, _D, C.c_int, C.c_int, _D]
        L.orc_speed_violated.argtypes = [_P, C.c_double, C.c_int]
        L.orc_speed_violated.restype = C.c_int
        L.orc_mlp.argtypes = [_P, _D, _D, _D]
        L.orc_controls.argtypes = [_P, _D, _D, _D]
        L.orc_euler_step.argtypes = [_P, _D, _D, _D]
        L.orc_collide.argtypes = [_P, C.c_double, C.c_double, C.c_double, _D, C.c_int,
                                  C.c_double, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_collide.restype = C.c_int
        L.orc_step.argtypes = [_P, _D, _D, _D, _D, C.c_int, C.c_int, _D, _D]
        L.orc_cost.argtypes = [_P, _D, _D, C.c_int, _D]
        L.orc_cost.restype = C.c_double
        L.orc_rollout_theta.argtypes = [_P, _D, C.c_int, _D, _D, _D, _D, C.c_int, C.c_int,
                                        C.c_int, _D, _I, C.c_void_p, C.c_void_p]
        L.orc_rollout_samples.argtypes = [_P, C.c_uint64, C.c_uint32, C.c_uint32, _I, C.c_int,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_uint32,
                                          _D, _D, _D, _D, C.c_int, C.c_int, C.c_int,
                                          _D, _I, C.c_void_p, C.c_void_p]
        L.orc_plan.argtypes = [_P, _D, _D, _D, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_uint32, C.c_int, _D, _I,
                               C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), C.POINTER(C.c_double), _D, _D, _D]
        L.orc_plan.restype = C.c_int
        L.orc_theta_mixed.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_void_p, C.c_void_p,
                                      C.c_int, C.c_uint32, _F]
        _lib = L
    return _lib


def _d(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ----------------------------------------------------------------- sampler
def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def u24(w):
    return lib().orc_u24(int(w))


def ln32(u):
    return lib().orc_ln32(float(u))


def sincos2pi32(K):
    s, c = C.c_float(), C.c_float()
    lib().orc_sincos2pi32(int(K), C.byref(s), C.byref(c))
    return s.value, c.value


def normal_pair(a, b):
    out = np.zeros(2, np.float32)
    lib().orc_normal_pair(int(a), int(b), out)
    return out


def theta(seed, t_index, n, n_theta, stream=0):
    """FP32 parameters of sample n (Philox + Normal32)."""
    out = np.zeros(n_theta, np.float32)
    lib().orc_theta(int(seed), int(t_index), int(stream), int(n), int(n_theta), out)
    return out


def theta_mixed(seed, t_index, n, n_theta, mu, sigma, n_prop, prop_stream=1):
    """FP32 parameters of sample n of a plan step with a proposal."""
    out = np.zeros(n_theta, np.float32)
    mu32, sg32 = _f32(mu), _f32(sigma)
    lib().orc_theta_mixed(int(seed), int(t_index), int(n), int(n_theta), _ptr(mu32), _ptr(sg32),
                          int(n_prop), int(prop_stream), out)
    return out


def n_theta(p):
    return lib().orc_n_theta(C.byref(make_config(p)))


# ----------------------------------------------------------------- pieces
def frame_to_ev(state_w, goal_w, obs_w):
    obs_w = _d(obs_w).reshape(-1, 4)
    M = obs_w.shape[0]
    goal_ev = np.zeros(4)
    obs_ev = np.zeros((max(M, 1), 4))
    lib().orc_frame_to_ev(_d(state_w, 6), _d(goal_w, 4), obs_w if M else np.zeros((1, 4)),
                          M, goal_ev, obs_ev)
    return goal_ev, obs_ev[:M]


def features(p, z, ap, goal_ev, h, T):
    s = np.zeros(16)
    lib().orc_features(C.byref(make_config(p)), _d(z, 4), _d(ap, 2), _d(goal_ev, 4), h, T, s)
    return s[: p["widths"][0]]


def speed_violated(p, v, h):
    """Whether state h with speed v discards the sample (speed limits on, h >= 1)."""
    return bool(lib().orc_speed_violated(C.byref(make_config(p)), float(v), int(h)))


def mlp(p, th, s):
    a = np.zeros(2)
    s16 = np.zeros(16)
    s16[: len(s)] = s
    lib().orc_mlp(C.byref(make_config(p)), _d(th), s16, a)
    return a


def controls(p, a_raw, ap):
    out = np.zeros(2)
    lib().orc_controls(C.byref(make_config(p)), _d(a_raw, 2), _d(ap, 2), out)
    return out


def euler_step(p, z, a):
    zn = np.zeros(4)
    lib().orc_euler_step(C.byref(make_config(p)), _d(z, 4), _d(a, 2), zn)
    return zn


def collide(p, x, y, phi, obs_ev, tau=0.0, margin=0.0):
    """(flag, n_clearly_inside, n_within_margin_of_a_face)."""
    obs_ev = _d(obs_ev).reshape(-1, 4)
    M = obs_ev.shape[0]
    nc, nn = C.c_int(), C.c_int()
    f = lib().orc_collide(C.byref(make_config(p)), float(x), float(y), float(phi),
                          obs_ev if M else np.zeros((1, 4)), M, float(tau), float(margin),
                          C.byref(nc), C.byref(nn))
    return bool(f), nc.value, nn.value


def step(p, th, z, ap, goal_ev, h, T):
    a = np.zeros(2)
    zn = np.zeros(4)
    lib().orc_step(C.byref(make_config(p)), _d(th), _d(z, 4), _d(ap, 2), _d(goal_ev, 4),
                   int(h), int(T), a, zn)
    return a, zn


def cost(p, zT, ctrl, goal_ev):
    """Cost of a collision-free rollout from its final EV-frame state zT and
    its applied controls ctrl [T][2] (the rollout's cost formula)."""
    ctrl = _d(ctrl).reshape(-1, 2)
    return lib().orc_cost(C.byref(make_config(p)), _d(zT, 4), ctrl, ctrl.shape[0], _d(goal_ev, 4))


# ----------------------------------------------------------------- rollouts
def rollout_theta(p, thetas, z0, ap0, goal_ev, obs_ev, T, n_threads=0, record=True):
    c = make_config(p)
    nt = lib().orc_n_theta(C.byref(c))
    thetas = _d(thetas).reshape(-1, nt)
    K = thetas.shape[0]
    obs_ev = _d(obs_ev).reshape(-1, 4)
    M = obs_ev.shape[0]
    cost = np.zeros(K)
    fh = np.zeros(K, np.int32)
    traj = np.zeros((K, T + 1, 4)) if record else None
    ctrl = np.zeros((K, T, 2)) if record else None
    lib().orc_rollout_theta(C.byref(c), thetas, K, _d(z0, 4), _d(ap0, 2), _d(goal_ev, 4),
                            obs_ev if M else np.zeros((1, 4)), M, T, n_threads, cost, fh,
                            _ptr(traj), _ptr(ctrl))
    return dict(cost=cost, first_hit=fh, traj=traj, ctrl=ctrl)


def rollout_samples(p, seed, t_index, idx, z0, ap0, goal_ev, obs_ev, T, warm=None,
                    stream=0, n_threads=0, record=True, mu=None, sigma=None, n_prop=0, prop_stream=1):
    """Rollouts of the sampled parameter vectors idx; with a proposal (mu,
    sigma FP32 arrays of n_theta) samples idx < n_prop are mu + sigma*eps."""
    c = make_config(p)
    idx = np.ascontiguousarray(idx, np.int32)
    K = idx.size
    obs_ev = _d(obs_ev).reshape(-1, 4)
    M = obs_ev.shape[0]
    cost = np.zeros(K)
    fh = np.zeros(K, np.int32)
    traj = np.zeros((K, T + 1, 4)) if record else None
    ctrl = np.zeros((K, T, 2)) if record else None
    w = None if warm is None else _d(warm)
    mu32, sg32 = _f32(mu), _f32(sigma)
    lib().orc_rollout_samples(C.byref(c), int(seed), int(t_index), int(stream), idx, K, _ptr(w),
                              _ptr(mu32), _ptr(sg32), int(n_prop), int(prop_stream),
                              _d(z0, 4), _d(ap0, 2), _d(goal_ev, 4),
                              obs_ev if M else np.zeros((1, 4)), M, T, n_threads, cost, fh,
                              _ptr(traj), _ptr(ctrl))
    return dict(cost=cost, first_hit=fh, traj=traj, ctrl=ctrl)


def plan(p, state_w, goal_w, obs_w, N, T, seed, t_index, warm=None, n_threads=0, mu=None,
         sigma=None, n_prop=0, prop_stream=1):
    c = make_config(p)
    nt = lib().orc_n_theta(C.byref(c))
    obs_w = _d(obs_w).reshape(-1, 4)
    M = obs_w.shape[0]
    costs = np.zeros(N)
    fh = np.zeros(N, np.int32)
    bi, st, bc = C.c_int32(), C.c_int32(), C.c_double()
    bt = np.zeros(nt)
    ctrl = np.zeros((T, 2))
    traj = np.zeros((T + 1, 4))
    w = None if warm is None else _d(warm, nt)
    rc = lib().orc_plan(C.byref(c), _d(state_w, 6), _d(goal_w, 4),
                        obs_w if M else np.zeros((1, 4)), M, N, T, int(seed), int(t_index),
                        _ptr(w), _ptr(_f32(mu)), _ptr(_f32(sigma)), int(n_prop), int(prop_stream), n_threads,
                        costs, fh, C.byref(bi), C.byref(st), C.byref(bc),
                        bt, ctrl, traj)
    if rc == 1:
        raise ValueError("invalid plan arguments")
    return dict(costs=costs, first_hit=fh, best_idx=bi.value, status=st.value,
                best_cost=bc.value, best_theta=bt, controls=ctrl, traj=traj)


def plan_tshc(p, state_w, goal_w, obs_w, N, T, seed, t_index, n_restarts, sigma_pert, warm=None, n_threads=0):
    """The hill climb's sampling loop (Sect. II-D): round 0 is `plan`; round
    r >= 1 keeps the best so far as sample 0 and draws the others as
    theta_best + sigma_pert eps (normals of Philox stream r).  Returns the
    final round's result and the best cost after every round."""
    nt = n_theta(p)
    r = plan(p, state_w, goal_w, obs_w, N, T, seed, t_index, warm=warm, n_threads=n_threads)
    history = [r["best_cost"]]
    sig = np.full(nt, np.float32(sigma_pert), np.float32)
    for k in range(1, n_restarts):
        best = r["best_theta"].astype(np.float32)
        r = plan(p, state_w, goal_w, obs_w, N, T, seed, t_index, warm=best.astype(np.float64),
                 n_threads=n_threads, mu=best, sigma=sig, n_prop=N, prop_stream=k)
        history.append(r["best_cost"])
    r["history"] = history
    return r
