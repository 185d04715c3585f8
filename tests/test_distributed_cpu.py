"""Multi-rank seam on CPU with gloo, world size 2: walker shards, the global
clipping window and the gradient all-reduce reproduce the single-process
result, for the helpers alone and for the VMC trainer's whole step."""

import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_08423_gb300 import distributed as pd


def _clip(E, out, cot, q=5.0):
    """This test's own statement of the clipping rule (Methods, ansatz
    optimisation): median m, mean absolute deviation d, logarithmic growth
    outside m +- q d; loss weights 2 (E' - mean E') / W."""
    e = E.numpy()
    m = np.median(e)
    Lq = q * np.mean(np.abs(e - m))
    x = e - m
    c = np.where(np.abs(x) > Lq, m + np.sign(x) * Lq * (1 + np.log(np.maximum(np.abs(x), 1e-300) / Lq)), e)
    out.copy_(torch.as_tensor(c))
    cot.copy_(torch.as_tensor(2 * (c - c.mean()) / len(c)))




def _worker(rank, world, port, E_all, G, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = pd.shard(len(E_all), rank, world)
    Ec, cot, loss = pd.global_clip(torch.as_tensor(E_all[lo:hi]), _clip)
    g = torch.as_tensor(G[lo:hi].T @ cot.numpy())  # this rank's partial gradient sum_w cot_w g_w
    pd.allreduce_grad(g)
    q.put((rank, lo, hi, Ec.numpy(), cot.numpy(), float(loss), g.numpy()))
    dist.destroy_process_group()


def test_sharded_clip_and_gradient_match_single_process():
    rng = np.random.default_rng(0)
    W = 1001
    E = np.concatenate([rng.normal(-14.6, 0.3, W - 3), [40.0, -80.0, 300.0]])
    G = rng.normal(size=(W, 7))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + int(rng.integers(0, 2000))
    procs = [ctx.Process(target=_worker, args=(r, 2, port, E, G, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref_c_t, ref_cot_t = torch.empty(W, dtype=torch.float64), torch.empty(W, dtype=torch.float64)
    _clip(torch.as_tensor(E), ref_c_t, ref_cot_t)
    ref_c, ref_cot = ref_c_t.numpy(), ref_cot_t.numpy()
    # the test's clipping rule agrees with the oracle's
    from oracle import clip as oclip
    np.testing.assert_allclose(ref_c, oclip.clip_local_energy(E), rtol=1e-15)
    ref_g = G.T @ ref_cot
    for rank, lo, hi, Ec, cot, loss, g in out:
        np.testing.assert_allclose(Ec, ref_c[lo:hi], rtol=1e-15)
        np.testing.assert_allclose(cot, ref_cot[lo:hi], rtol=1e-14, atol=1e-18)
        np.testing.assert_allclose(loss, ref_c.mean(), rtol=1e-14)
        np.testing.assert_allclose(g, ref_g, rtol=1e-12, atol=1e-14)
    assert sorted((lo, hi) for _, lo, hi, *_ in out) == [(0, 501), (501, 1001)]


def test_shard_covers_every_walker_once():
    for W in (1, 7, 4096, 4099):
        for world in (1, 2, 3, 8):
            ranges = [pd.shard(W, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == W
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))


# ------------------------------------------------------------ trainer step

class _ToySystem:
    """A stand-in for a system handle on the CPU: one electron, ln psi =
    theta . f(r) with fixed features f, E_loc = sum_k theta_k^2 f_k(r) +
    |r|^2 / 2, a sampler that leaves the walkers in place (so that sharded
    and unsharded runs see the same configurations)."""

    P = 5
    N = 1

    def __init__(self):
        self.n_params = self.P
        self.theta = torch.zeros(self.P, dtype=torch.float64)

    def _f(self, r):
        x = r[:, 0, :]
        k = torch.arange(1, self.P + 1, dtype=torch.float64) / self.P
        return torch.exp(-k * (x * x).sum(-1, keepdim=True)) * (1 + k * x[:, :1])

    def set_params(self, th):
        self.theta = th.clone()

    def eval_logpsi(self, r, lp, sg):
        lp.copy_(self._f(r) @ self.theta)
        sg.fill_(1.0)

    def metropolis_step(self, r, lp, n, sigma, seed, step0):
        pass

    def eval_local_energy(self, r, E):
        E.copy_(self._f(r) @ (self.theta ** 2) + 0.5 * (r[:, 0, :] ** 2).sum(-1))

    def grad_logpsi(self, r, cot, out, mem_budget_bytes=0):
        out.copy_(self._f(r).T @ cot)


def _adamw(theta, g, m, v, lr, t, b1, b2, eps, wd):
    m.mul_(b1).add_((1 - b1) * g)
    v.mul_(b2).add_((1 - b2) * g * g)
    theta.sub_(lr * (m / (1 - b1 ** t) / (torch.sqrt(v / (1 - b2 ** t)) + eps) + wd * theta))


def _train(r0, steps, group=None):
    from paper_1909_08423_gb300.vmc import VMCTrainer
    rank = dist.get_rank() if dist.is_initialized() else 0
    world = dist.get_world_size() if dist.is_initialized() else 1
    lo, hi = pd.shard(len(r0), rank, world)
    tr = VMCTrainer(_ToySystem(), np.linspace(-0.3, 0.4, _ToySystem.P), walkers=len(r0), batch=2 * len(r0),
                    resample_period=3, n_discard=1, n_decorr=1, lr=0.05, device="cpu", group=group,
                    kernels={"clip": _clip, "adamw": _adamw}, r0=r0[lo:hi])
    hist = [tr.step()["loss"] for _ in range(steps)]
    return tr.theta.numpy(), hist


def _trainer_worker(rank, world, port, r0, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    theta, hist = _train(r0, 4)
    q.put((rank, theta, hist))
    dist.destroy_process_group()


def test_trainer_step_on_two_ranks_matches_one():
    """Four training steps (pool refill, clipped loss gradient, AdamW) on two
    gloo ranks holding half of the walkers each give the parameters and
    losses of one process holding all of them."""
    rng = np.random.default_rng(4)
    r0 = rng.normal(size=(64, 1, 3))
    r0[3] *= 6.0  # outliers for the clipping window
    theta1, hist1 = _train(r0, 4)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + int(rng.integers(0, 2000))
    procs = [ctx.Process(target=_trainer_worker, args=(r, 2, port, r0, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, theta, hist in out:
        np.testing.assert_allclose(theta, theta1, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(hist, hist1, rtol=1e-12)
