"""Multi-rank seam on CPU with gloo, world size 2: walker shards, the global
clipping window and the gradient all-reduce reproduce the single-process
result."""

import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import clip as oclip
from paper_1909_08423_gb300 import distributed as pd


def _oracle_clip(E, out, cot):
    e = E.numpy()
    c = oclip.clip_local_energy(e)
    out.copy_(torch.as_tensor(c))
    cot.copy_(torch.as_tensor(oclip.loss_cotangent(c)))


def _worker(rank, world, port, E_all, G, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = pd.shard(len(E_all), rank, world)
    Ec, cot, loss = pd.global_clip(torch.as_tensor(E_all[lo:hi]), _oracle_clip)
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
    ref_c = oclip.clip_local_energy(E)
    ref_cot = oclip.loss_cotangent(ref_c)
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
