"""VMC training driver (Methods, ansatz optimisation; hyperparameter table).

Every numeric step runs in the library's kernels; this module only orders
them.  One training step takes the next batch of a pool of sampled
configurations, forms the clipped local energies and the loss gradient
sum_w 2 (E_w - L) / W grad ln|psi_w| (Eq. trainig), applies AdamW with the
decaying learning rate lr0 / (1 + t / t0) and uploads the new parameters.
Every `resample_period` steps the pool is refilled from the current wave
function: the chains continue from their last positions, `n_discard` steps
are thrown away, then `walkers` configurations are collected every
`n_decorr` steps until the pool holds resample_period x batch of them, so
that each configuration is used once.  Defaults are the paper's table
(batch 10000, 2000 walkers, resampling period 100, 50 discarded and 1
decorrelation step, lr 0.01, t0 = 200, clipping window 5).
"""

from __future__ import annotations

import torch

from . import binding, checkpoint
from . import distributed as pd
from .autograd import vmc_loss_and_grad


class VMCTrainer:
    """Under torch.distributed (one process per GPU) each rank holds its
    shard of the walkers and of every batch; its chains draw from the Philox
    key seed + rank; the clipping window, the loss and the gradient are taken
    over all ranks (see vmc_loss_and_grad), so every rank applies the same
    AdamW update and the parameters stay identical.  `kernels` may replace
    the library's clipping and AdamW calls (clip(E, Ec, cot), adamw(theta,
    grad, m, v, lr, t, b1, b2, eps, wd)); `r0` gives this rank's initial
    walkers instead of pn_init_walkers."""

    def __init__(self, system, params, walkers=2000, batch=10000, resample_period=100, n_discard=50, n_decorr=1,
                 lr=0.01, t0=200.0, weight_decay=0.01, betas=(0.9, 0.999), eps=1e-8, q=5.0, sampler="metropolis",
                 sigma=0.2, tau=0.1, seed=0, device="cuda", group=None, kernels=None, r0=None):
        if sampler not in ("metropolis", "langevin"):
            raise ValueError("sampler must be 'metropolis' or 'langevin'")
        self.s = system
        self.group = group
        self.world, self.rank = pd.world_size(group), pd.rank_of(group)
        k = kernels or {}
        self._clip = k.get("clip") or (lambda E, Ec, cot: binding.clip_local_energy(E, Ec, cot, q))
        self._adamw = k.get("adamw") or binding.adamw_step
        self.theta = torch.as_tensor(params, dtype=torch.float64, device=device).clone().contiguous()
        if self.theta.numel() != system.n_params:
            raise ValueError(f"{self.theta.numel()} parameters given, the system has {system.n_params}")
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.cfg = dict(walkers=walkers, batch=batch, resample_period=resample_period, n_discard=n_discard,
                        n_decorr=n_decorr, lr=lr, t0=t0, weight_decay=weight_decay, betas=betas, eps=eps, q=q,
                        sampler=sampler, sigma=sigma, tau=tau, seed=seed)
        lo, hi = pd.shard(walkers, self.rank, self.world)
        blo, bhi = pd.shard(batch, self.rank, self.world)
        self.W_local, self.B_local = hi - lo, bhi - blo
        self.seed_local = seed + self.rank
        self.t = 0
        self.mc_step = 0
        N = system.N
        self.r = torch.empty(self.W_local, N, 3, dtype=torch.float64, device=device)
        system.set_params(self.theta)
        if r0 is not None:
            self.r.copy_(torch.as_tensor(r0, dtype=torch.float64))
        else:
            system.init_walkers(self.r, self.seed_local)
        self.lp = torch.empty(self.W_local, dtype=torch.float64, device=device)
        self.drift = torch.empty_like(self.r) if sampler == "langevin" else None
        n_pool = resample_period * self.B_local
        self.pool = torch.empty(n_pool, N, 3, dtype=torch.float64, device=device)

    def _advance(self, n):
        c = self.cfg
        if n <= 0:
            return
        if c["sampler"] == "metropolis":
            self.s.metropolis_step(self.r, self.lp, n, c["sigma"], self.seed_local, self.mc_step)
        else:
            self.s.langevin_step(self.r, self.lp, self.drift, n, c["tau"], self.seed_local, self.mc_step)
        self.mc_step += n

    def resample(self):
        """Refill the pool from the current parameters."""
        c = self.cfg
        if c["sampler"] == "metropolis":
            sg = torch.empty_like(self.lp)
            self.s.eval_logpsi(self.r, self.lp, sg)
        else:
            self.s.eval_drift(self.r, self.drift, self.lp)
        self._advance(c["n_discard"])
        n_pool, W = self.pool.shape[0], self.W_local
        filled = 0
        while filled < n_pool:
            self._advance(c["n_decorr"])
            k = min(W, n_pool - filled)
            self.pool[filled:filled + k].copy_(self.r[:k])
            filled += k

    def step(self):
        """One optimisation step; returns the clipped loss and batch statistics."""
        c = self.cfg
        if self.t % c["resample_period"] == 0:
            self.resample()
        k = self.t % c["resample_period"]
        rb = self.pool[k * self.B_local:(k + 1) * self.B_local]
        loss, grad, E = vmc_loss_and_grad(self.s, rb, c["q"], clip_fn=self._clip, group=self.group)
        lr = c["lr"] / (1.0 + self.t / c["t0"])
        self._adamw(self.theta, grad, self.m, self.v, lr, self.t + 1, c["betas"][0], c["betas"][1], c["eps"],
                    c["weight_decay"])
        self.s.set_params(self.theta)
        self.t += 1
        fin = torch.isfinite(E)
        Ef = E[fin]
        return {"step": self.t, "loss": float(loss), "e_mean": float(Ef.mean()),
                "e_stderr": float(Ef.std() / max(1, Ef.numel()) ** 0.5), "lr": lr}

    # ------------------------------------------------------ checkpointing
    def save(self, path):
        """Everything the next steps depend on (parameters, AdamW moments,
        step counters, walkers and their RNG position, the sampled pool)."""
        checkpoint.save(path, {"theta": self.theta, "m": self.m, "v": self.v, "r": self.r, "lp": self.lp,
                               "drift": self.drift, "pool": self.pool},
                        {"kind": "vmc", "t": self.t, "mc_step": self.mc_step,
                         "cfg": {k: list(v) if isinstance(v, tuple) else v for k, v in self.cfg.items()}})

    def load(self, path):
        a, m = checkpoint.load(path, device=self.theta.device)
        if m.get("kind") != "vmc":
            raise ValueError(f"{path}: holds {m.get('kind')}, not a training state")
        cfg = {k: tuple(v) if isinstance(v, list) else v for k, v in m["cfg"].items()}
        if cfg != self.cfg:
            raise ValueError("checkpoint was written with another training configuration")
        for k in ("theta", "m", "v", "r", "lp", "pool"):
            getattr(self, k).copy_(a[k])
        if self.drift is not None:
            self.drift.copy_(a["drift"])
        self.t, self.mc_step = m["t"], m["mc_step"]
        self.s.set_params(self.theta)
