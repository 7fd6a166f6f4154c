"""Learned sampling proposal: data from the planner, training and
evaluation, driven over the C ABI (every step runs in the library's
kernels: plan steps, scene encoding, the tensor-core network, Adam).

Data: (scene encoding, best-found parameters) pairs on course-like scenes
(inputs.scene_proposal_batch).  Training: Gaussian negative log-likelihood
of the best parameters under the proposal, Adam.

Two ways to make the pairs:
* `generate`: the plain isotropic sampler's winners.  Measured on GB300,
  these do not train a useful diagonal Gaussian: the winners' hidden-layer
  parameters are independent random draws, so their per-parameter
  distribution given the scene stays close to N(0, 1) (even the elite
  samples of a scene, fitted per scene, have a standard deviation of 0.99).
* `bootstrap` (the training recipe): expert iteration in a fixed parameter
  basis.  The untrained proposal is N(theta_0, 0.3^2 I) for a fixed random
  theta_0; each round plans fresh scenes with the mixed plan step (the
  proposal's samples plus isotropic ones, every sample judged by the exact
  rollout cost, so the isotropic sampler still wins whenever it finds the
  better plan) and trains on the scenes whose winner came from the
  proposal.  The winners then share theta_0's basis and the network learns
  scene-dependent shifts of it.

Evaluation: per held-out scene, the plain plan step with N samples against
the mixed plan step with N and with N/4 samples.
"""
import math

import numpy as np
import torch

from . import inputs, npp

N_THETA = 450
N_IN = 72


def _scene_array(scenes):
    return npp.make_scenes(scenes)


class ProposalNet:
    """The network on one device (a thin owner of an npp_proposal)."""

    def __init__(self, batch=1024, device=0, ls_min=-3.0, ls_max=1.0):
        self.batch = batch
        self.device = torch.device("cuda", device)
        self.P = npp.npp_proposal_create(batch, ls_min=ls_min, ls_max=ls_max, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    def init(self, seed, out_scale=0.01, base=None, base_std=1.0):
        """He-normal hidden layers, small output layer: the untrained
        proposal is N(base, base_std^2 I) for every scene (base 0 and std 1
        by default, the isotropic sampler)."""
        rng = np.random.default_rng(seed)
        H, O = 256, 2 * N_THETA
        b3 = np.zeros(O)
        if base is not None:
            b3[:N_THETA] = base
        b3[N_THETA:] = math.log(base_std)
        parts = [rng.standard_normal((H, N_IN)) * math.sqrt(2.0 / N_IN), np.zeros(H),
                 rng.standard_normal((H, H)) * math.sqrt(2.0 / H), np.zeros(H),
                 rng.standard_normal((O, H)) * out_scale * math.sqrt(1.0 / H), b3]
        self.set_params(np.concatenate([p.ravel() for p in parts]))

    def set_params(self, vec):
        npp.npp_proposal_set_params(self.P, vec)

    def params(self):
        return npp.npp_proposal_get_params(self.P)

    def grads(self):
        return npp.npp_proposal_get_grads(self.P)

    def forward(self, x):
        """x: CUDA float32 [n][72], n <= batch -> (mean, std) [n][450]."""
        n = x.shape[0]
        mean = torch.empty(n, N_THETA, dtype=torch.float32, device=self.device)
        std = torch.empty_like(mean)
        npp.npp_proposal_forward(self.P, x.contiguous(), n, mean, std)
        return mean, std

    def train_step(self, x, theta, lr):
        npp.npp_proposal_train_step(self.P, x.contiguous(), theta.contiguous(), lr, self.loss)
        return self.loss

    def close(self):
        if self.P is not None:
            npp.npp_proposal_destroy(self.P)
            self.P = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode(planner, scenes, obs_dev):
    """Scene encodings [S][72] on the device."""
    arr = _scene_array(scenes)
    sd = npp.scenes_to_device(arr, planner.device.index or 0)
    x = torch.empty(len(scenes), N_IN, dtype=torch.float32, device=planner.device)
    npp.npp_proposal_encode(planner.h, sd, len(scenes), obs_dev, x)
    return x


def plain_best(planner, scenes, obs_dev):
    """Best parameters, costs and status of every scene by the plain
    isotropic sampler (one batched plan)."""
    S = len(scenes)
    arr = _scene_array(scenes)
    B = npp.npp_batch_create(planner.h, arr)
    off = npp.npp_batch_offsets(B, S)
    dev = planner.device
    best = torch.zeros(S, 8, dtype=torch.int32, device=dev)
    params = torch.zeros(int(off[S, 0]), dtype=torch.float32, device=dev)
    controls = torch.zeros(int(off[S, 1]) * 2, dtype=torch.float32, device=dev)
    traj = torch.zeros(int(off[S, 2]) * 4, dtype=torch.float32, device=dev)
    out = npp.npp_batch_outputs()
    out.best = best.data_ptr()
    out.params = params.data_ptr()
    out.controls = controls.data_ptr()
    out.trajectory = traj.data_ptr()
    npp.npp_plan_batch(B, obs_dev, out)
    torch.cuda.synchronize()
    npp.npp_batch_destroy(B)
    b = best.cpu()
    cost = b[:, 2].view(torch.float32).numpy().copy()
    status = b[:, 1].numpy().copy()
    theta = params.view(S, N_THETA)
    return theta, cost, status


def generate(seed, S, N=4096, T=40, chunk=512, device=0, n_layouts=16):
    """S (encoding, best theta) pairs; rows whose plain plan was infeasible
    are dropped.  Returns CUDA tensors X [S'][72], Theta [S'][450] and the
    plain costs."""
    Xs, Ts, Cs = [], [], []
    planner = None
    for c0 in range(0, S, chunk):
        b = inputs.scene_proposal_batch(seed * 100003 + c0 // chunk, S=min(chunk, S - c0), N=N, T=T,
                                        n_layouts=n_layouts)
        if planner is None:
            planner = npp.Planner(b["preset"], max_N=N, max_T=T, max_M=b["obs"].shape[0], device=device)
        obs = torch.tensor(b["obs"], dtype=torch.float32, device=planner.device)
        x = encode(planner, b["scenes"], obs)
        th, cost, status = plain_best(planner, b["scenes"], obs)
        ok = torch.from_numpy(status == 0).to(planner.device)
        Xs.append(x[ok])
        Ts.append(th[ok])
        Cs.append(cost[status == 0])
    planner.close()
    return torch.cat(Xs), torch.cat(Ts), np.concatenate(Cs)


def train(net, X, Theta, epochs=10, lr=1e-3, seed=0, lr_final=None):
    """Adam on shuffled full batches; returns the mean loss per epoch."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    B = net.batch
    steps = max(1, n // B)
    hist = []
    total = epochs * steps
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        acc = torch.zeros(1, device=X.device)
        for s in range(steps):
            idx = perm[s * B:(s + 1) * B]
            rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, total - 1))
            acc += net.train_step(X[idx], Theta[idx], rate)
            k += 1
        hist.append(float(acc.item()) / steps)
    return hist


def plan_costs(planner, scenes, obs_dev, N, mean=None, std=None, N_prop=0, params_out=None):
    """Best cost (inf if infeasible) of each scene's plan step: plain when
    mean is None, else mixed with N_prop proposal samples.  params_out
    (CUDA [S][450]) receives each winner's parameters."""
    out = planner.outputs()
    costs = np.zeros(len(scenes))
    winners = np.zeros(len(scenes), np.int64)
    for i, sc in enumerate(scenes):
        o = obs_dev[sc["obs_offset"]:sc["obs_offset"] + sc["M"]]
        if mean is None:
            npp.npp_plan_step(planner.h, sc["state"], sc["goal"], o, sc["M"], N, sc["T"], sc["seed"], 0,
                              None, out)
        else:
            npp.npp_plan_step_proposal(planner.h, sc["state"], sc["goal"], o, sc["M"], N, sc["T"], sc["seed"],
                                       0, None, mean[i], std[i], N_prop, out)
        if params_out is not None:
            params_out[i].copy_(planner.params)
        b = planner.best.cpu()
        st = int(b[1])
        costs[i] = b[2:3].view(torch.float32).item() if st == 0 else np.inf
        winners[i] = int(b[0])
    return costs, winners


def bootstrap(net, rounds=4, S=8192, N=4096, T=40, prop_frac=0.5, epochs=8, lr=1e-3, seed=0,
              device=0, only_proposal_winners=False, log=None):
    """Expert iteration: each round plans S fresh scenes with the mixed
    planner (the current proposal's samples plus isotropic ones, every
    sample judged by the exact rollout cost; round 0 with an untrained
    proposal), and trains on (encoding, winner parameters) pairs.  Returns
    per-round statistics."""
    stats = []
    for r in range(rounds):
        b = inputs.scene_proposal_batch(seed * 7919 + 31 * r + 1, S=S, N=N, T=T)
        planner = npp.Planner(b["preset"], max_N=N, max_T=T, max_M=b["obs"].shape[0], device=device)
        obs = torch.tensor(b["obs"], dtype=torch.float32, device=planner.device)
        x = encode(planner, b["scenes"], obs)
        means, stds = [], []
        for c0 in range(0, S, net.batch):
            m, sd = net.forward(x[c0:c0 + net.batch])
            means.append(m.clone())
            stds.append(sd.clone())
        mean, std = torch.cat(means), torch.cat(stds)
        theta = torch.zeros(S, N_THETA, dtype=torch.float32, device=planner.device)
        npr = int(prop_frac * N)
        costs, win = plan_costs(planner, b["scenes"], obs, N, mean, std, npr, params_out=theta)
        planner.close()
        keep = np.isfinite(costs)
        if only_proposal_winners:
            keep &= win < npr
        kt = torch.from_numpy(keep).to(x.device)
        hist = train(net, x[kt], theta[kt], epochs=epochs, lr=lr, seed=seed + r)
        st = dict(round=r, mean_cost=float(np.mean(costs[np.isfinite(costs)])),
                  proposal_won=float(np.mean(win[np.isfinite(costs)] < npr)), n_train=int(keep.sum()),
                  loss_first=hist[0], loss_last=hist[-1], mean_std=float(std.mean()))
        stats.append(st)
        if log:
            log(st)
    return stats


def train_proposal(rounds=30, S=8192, N=2048, T=40, epochs=4, lr=1e-3, base_seed=123, base_std=0.3,
                   batch=1024, seed=0, device=0, log=None):
    """The training recipe: a fresh network around a fixed random basis
    theta_0 (Philox-independent numpy draw from base_seed), then `rounds`
    rounds of expert iteration on proposal-won scenes."""
    net = ProposalNet(batch=batch, device=device)
    base = np.random.default_rng(base_seed).standard_normal(N_THETA)
    net.init(seed, base=base, base_std=base_std)
    stats = bootstrap(net, rounds=rounds, S=S, N=N, T=T, prop_frac=0.5, epochs=epochs, lr=lr, seed=seed,
                      device=device, only_proposal_winners=True, log=log)
    return net, stats


def evaluate(net, seed, S=256, Ns=(512, 2048, 8192), prop_frac=0.5, device=0, T=40):
    """Held-out scenes: plain with N samples vs mixed with N and with N/4
    samples (prop_frac of them from the proposal).  Returns per-N mean
    costs over scenes feasible in all arms and the proposal-win rates."""
    b = inputs.scene_proposal_batch(10 ** 6 + seed, S=S, N=max(Ns), T=T)
    planner = npp.Planner(b["preset"], max_N=max(Ns), max_T=T, max_M=b["obs"].shape[0], device=device)
    obs = torch.tensor(b["obs"], dtype=torch.float32, device=planner.device)
    x = encode(planner, b["scenes"], obs)
    means, stds = [], []
    for c0 in range(0, S, net.batch):
        m, s = net.forward(x[c0:c0 + net.batch])
        means.append(m)
        stds.append(s)
    mean, std = torch.cat(means), torch.cat(stds)
    res = {}
    for N in Ns:
        plain, _ = plan_costs(planner, b["scenes"], obs, N)
        mixed, w = plan_costs(planner, b["scenes"], obs, N, mean, std, int(prop_frac * N))
        q = max(32, N // 4)
        mixed_q, wq = plan_costs(planner, b["scenes"], obs, q, mean, std, int(prop_frac * q))
        ok = np.isfinite(plain) & np.isfinite(mixed) & np.isfinite(mixed_q)
        res[N] = dict(plain=float(np.mean(plain[ok])), mixed=float(np.mean(mixed[ok])),
                      mixed_quarter=float(np.mean(mixed_q[ok])), n_scenes=int(ok.sum()),
                      proposal_won=float(np.mean(w[ok] < int(prop_frac * N))),
                      quarter_not_worse=float(np.mean(mixed_q[ok] <= plain[ok] + 1e-6)))
    planner.close()
    return res
