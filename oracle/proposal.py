"""FP64 oracle of the learned sampling proposal.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU
baseline of the benchmark may import this module; the CUDA library never
calls it and shares no code with it.

The paper samples the controller parameters theta isotropically (Sect. II-D
"Fourth": theta ~ N(0, I) per sampling time) and names guiding the sampling
with pre-encoded knowledge as future work (Sect. V).  The proposal built
here is that guide: a small network maps a scene encoding to the mean and
log standard deviation of a diagonal Gaussian over theta.  Its parts:

* scene encoding (72 inputs): a 64-bin polar histogram of the obstacle
  points in the EV-aligned frame at t (bin k covers headings
  [-pi + k 2pi/64, -pi + (k+1) 2pi/64)), each point weighted by its nearness
  max(0, 1 - d / 20 m), squashed as h / (1 + h); then the 8 network inputs
  s_t of the rollout at h = 0 (Eq. eq_def_stph and the three project
  features);
* network: 72 -> 256 (ReLU) -> 256 (ReLU) -> 900 = (mean, raw log-std) of
  the 450 parameters of the 8-16-16-2 controller; log-std clamped to
  [LS_MIN, LS_MAX];
* loss: Gaussian negative log-likelihood of the best-found parameters,
  averaged over batch and parameters (constant term dropped);
* optimiser: Adam (Kingma & Ba, ICLR 2015) with bias correction, FP64
  master weights here (FP32 on the device);
* arithmetic model of the device: inputs, weights, hidden activations and
  the output gradient are rounded to BF16 (round to nearest even) where the
  device stores them in BF16; all sums here are exact-ish FP64 (the device
  accumulates in FP32).  quantize=False gives the plain FP64 network, whose
  gradients are pinned by finite differences.
"""
import math

import numpy as np

NBINS = 64
R_HIST = 20.0
N_FEAT = 8
N_IN = NBINS + N_FEAT          # 72
HIDDEN = 256
N_THETA = 450                   # parameters of the 8-16-16-2 controller
N_OUT = 2 * N_THETA             # 900
LS_MIN = -3.0
LS_MAX = 1.0
SHAPES = (("W1", (HIDDEN, N_IN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (N_OUT, HIDDEN)), ("b3", (N_OUT,)))


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def pack(params):
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k, _ in SHAPES])


def unpack(vec):
    vec = np.asarray(vec, np.float64)
    out, o = {}, 0
    for k, s in SHAPES:
        n = int(np.prod(s))
        out[k] = vec[o:o + n].reshape(s).copy()
        o += n
    return out


def init_params(seed, out_scale=0.01):
    """He-normal hidden layers, a small output layer (mean ~ 0, log-std ~ 0:
    the untrained proposal is close to the isotropic sampler)."""
    rng = np.random.default_rng(seed)
    p = {}
    p["W1"] = rng.standard_normal((HIDDEN, N_IN)) * math.sqrt(2.0 / N_IN)
    p["b1"] = np.zeros(HIDDEN)
    p["W2"] = rng.standard_normal((HIDDEN, HIDDEN)) * math.sqrt(2.0 / HIDDEN)
    p["b2"] = np.zeros(HIDDEN)
    p["W3"] = rng.standard_normal((N_OUT, HIDDEN)) * out_scale * math.sqrt(1.0 / HIDDEN)
    p["b3"] = np.zeros(N_OUT)
    return p


def bf16(x):
    """Round to the nearest BF16 value (8 significant bits), ties to even."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0), e - 8)


# ------------------------------------------------------------------ encoding
def polar_hist(obs_ev, R=R_HIST, nbins=NBINS, margin=1e-4):
    """Nearness-weighted polar histogram of EV-frame points (rows x, y, ...).
    Returns (h[nbins], amb[nbins]): amb[k] is the total weight of points
    whose heading lies within `margin` bin widths of a boundary of bin k
    (such a point may fall on either side in another precision)."""
    obs_ev = np.asarray(obs_ev, np.float64).reshape(-1, 4)
    h = np.zeros(nbins)
    amb = np.zeros(nbins)
    for px, py in obs_ev[:, :2]:
        d = math.hypot(px, py)
        w = max(0.0, 1.0 - d / R)
        if w <= 0.0:
            continue
        u = (math.atan2(py, px) + math.pi) * (nbins / (2.0 * math.pi))
        k = min(int(math.floor(u)), nbins - 1)
        h[k] += w
        r = u - round(u)
        if abs(r) < margin:
            i = int(round(u))
            amb[i % nbins] += w
            amb[(i - 1) % nbins] += w
    return h, amb


def squash(h):
    return h / (1.0 + h)


def encode(p, state_w, goal_w, obs_w, T):
    """72-d scene encoding (histogram part squashed) and the histogram
    itself with its ambiguity weights."""
    from oracle import oracle as orc
    st = np.asarray(state_w, np.float64)
    goal_ev, obs_ev = orc.frame_to_ev(st, np.asarray(goal_w, np.float64),
                                      np.asarray(obs_w, np.float64).reshape(-1, 4))
    h, amb = polar_hist(obs_ev)
    s = orc.features(p, [0.0, 0.0, 0.0, st[3]], st[4:6], goal_ev, 0, T)
    return np.concatenate([squash(h), s]), h, amb


# ------------------------------------------------------------------ network
def forward(params, X, quantize=True):
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    X = np.asarray(X, np.float64).reshape(-1, N_IN)
    Xq = q(X)
    W1, W2, W3 = q(params["W1"]), q(params["W2"]), q(params["W3"])
    Z1 = Xq @ W1.T + params["b1"]
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + params["b2"]
    H2 = q(np.maximum(Z2, 0.0))
    Y = H2 @ W3.T + params["b3"]
    mu = Y[:, :N_THETA]
    raw = Y[:, N_THETA:]
    ls = np.clip(raw, LS_MIN, LS_MAX)
    return dict(Xq=Xq, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Y=Y, mu=mu, raw=raw, ls=ls, W1=W1, W2=W2, W3=W3)


def nll(cache, theta):
    """Mean over batch and parameters of log sigma + (theta - mu)^2 / (2 sigma^2)."""
    theta = np.asarray(theta, np.float64).reshape(cache["mu"].shape)
    r = theta - cache["mu"]
    return float(np.mean(cache["ls"] + 0.5 * r * r * np.exp(-2.0 * cache["ls"])))


def backward(params, cache, theta, quantize=True):
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    theta = np.asarray(theta, np.float64).reshape(cache["mu"].shape)
    B = theta.shape[0]
    scale = 1.0 / (B * N_THETA)
    r = theta - cache["mu"]
    e2 = np.exp(-2.0 * cache["ls"])
    dmu = -r * e2 * scale
    inside = (cache["raw"] > LS_MIN) & (cache["raw"] < LS_MAX)
    dls = (1.0 - r * r * e2) * scale * inside
    dY = q(np.concatenate([dmu, dls], axis=1))
    g = {}
    g["W3"] = dY.T @ cache["H2"]
    g["b3"] = dY.sum(0)
    dZ2 = q((dY @ cache["W3"]) * (cache["H2"] > 0))
    g["W2"] = dZ2.T @ cache["H1"]
    g["b2"] = dZ2.sum(0)
    dZ1 = q((dZ2 @ cache["W2"]) * (cache["H1"] > 0))
    g["W1"] = dZ1.T @ cache["Xq"]
    g["b1"] = dZ1.sum(0)
    return g


def adam_init():
    return dict(m=None, v=None, t=0)


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update with bias correction (Kingma & Ba, Algorithm 1)."""
    g = pack(grads)
    w = pack(params)
    m = np.zeros_like(w) if state["m"] is None else state["m"]
    v = np.zeros_like(w) if state["v"] is None else state["v"]
    t = state["t"] + 1
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    w = w - lr * mhat / (np.sqrt(vhat) + eps)
    return unpack(w), dict(m=m, v=v, t=t)


def mean_std(params, X, quantize=True):
    """Sampling proposal of each row of X: mean and standard deviation of
    the 450 parameters."""
    c = forward(params, X, quantize)
    return c["mu"], np.exp(c["ls"])
