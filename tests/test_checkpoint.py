"""Checkpoint files (CPU) and resumed runs that continue bit for bit (GPU)."""

import numpy as np
import pytest
import torch

from paper_1909_08423_gb300 import checkpoint, synth


def test_chain_file_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    r, lp, d = rng.normal(size=(7, 4, 3)), rng.normal(size=7), rng.normal(size=(7, 4, 3))
    p = tmp_path / "c.npz"
    checkpoint.save_chain(p, r, lp, seed=2 ** 63 + 5, next_step=12345678901, drift=d)
    c = checkpoint.load_chain(p, device="cpu")
    np.testing.assert_array_equal(c["r"].numpy(), r)
    np.testing.assert_array_equal(c["logabs"].numpy(), lp)
    np.testing.assert_array_equal(c["drift"].numpy(), d)
    assert c["seed"] == 2 ** 63 + 5 and c["next_step"] == 12345678901


def test_foreign_file_is_refused(tmp_path):
    p = tmp_path / "x.npz"
    np.savez(p, __meta__=np.frombuffer(b'{"format": "other"}', dtype=np.uint8))
    with pytest.raises(ValueError):
        checkpoint.load(p)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_metropolis_resumed_is_bitwise_uninterrupted(lib, tmp_path, precision):
    """100 Metropolis steps in one call equal 50 steps, a checkpoint written
    and read back into fresh buffers, and 50 more steps."""
    sysd = synth.be()
    W = 512
    s = lib.System(sysd, precision=precision, max_walkers=W)
    r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, 4)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    s.eval_logpsi(r, lp, sg)
    r1, lp1 = r.clone(), lp.clone()
    s.metropolis_step(r1, lp1, 100, 0.2, 9, 0)
    s.metropolis_step(r, lp, 50, 0.2, 9, 0)
    checkpoint.save_chain(tmp_path / "c.npz", r, lp, seed=9, next_step=50)
    del r, lp
    c = checkpoint.load_chain(tmp_path / "c.npz")
    s2 = lib.System(sysd, precision=precision, max_walkers=W)
    s2.metropolis_step(c["r"], c["logabs"], 100 - c["next_step"], 0.2, c["seed"], c["next_step"])
    torch.cuda.synchronize()
    assert torch.equal(c["r"], r1) and torch.equal(c["logabs"], lp1)


@pytest.mark.gpu
def test_training_resumed_is_bitwise_uninterrupted(lib, tmp_path):
    """Six optimisation steps in a row equal three, a checkpoint of the
    trainer, a new trainer loaded from it, and three more (same pool,
    parameters, AdamW moments and chain positions)."""
    from paper_1909_08423_gb300.vmc import VMCTrainer
    sysd = synth.h2()
    kw = dict(walkers=64, batch=128, resample_period=4, n_discard=5, n_decorr=1, seed=3)
    flat = synth.flatten_params(sysd)
    a = VMCTrainer(lib.System(sysd, precision=lib.PN_FP64, max_walkers=128), flat, **kw)
    for _ in range(6):
        a.step()
    b = VMCTrainer(lib.System(sysd, precision=lib.PN_FP64, max_walkers=128), flat, **kw)
    for _ in range(3):
        b.step()
    b.save(tmp_path / "t.npz")
    c = VMCTrainer(lib.System(sysd, precision=lib.PN_FP64, max_walkers=128), flat, **kw)
    c.load(tmp_path / "t.npz")
    for _ in range(3):
        c.step()
    torch.cuda.synchronize()
    assert torch.equal(a.theta, c.theta) and torch.equal(a.m, c.m) and torch.equal(a.v, c.v)
    assert torch.equal(a.r, c.r) and a.t == c.t and a.mc_step == c.mc_step
