"""VMC training through the library: the AdamW kernel against the oracle's
AdamW, and a short training run of H2 whose energy must fall and, by the
variational principle, stay above the exact ground-state energy."""

import numpy as np
import pytest
import torch

from oracle import optim
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

E_H2_EXACT = -1.1745  # Ha, H2 at a bond length of 1.4 bohr


def test_adamw_kernel_matches_oracle(lib):
    from paper_1909_08423_gb300 import binding
    rng = np.random.default_rng(2)
    n = 10001
    th = rng.normal(size=n)
    m = np.zeros(n)
    v = np.zeros(n)
    thd, md, vd = (torch.as_tensor(a, device="cuda").clone() for a in (th, m, v))
    for t in range(1, 8):
        g = rng.normal(size=n) * (10.0 ** rng.integers(-6, 2, size=n))
        lr = optim.learning_rate(t - 1, 0.01, 200)
        th, m, v = optim.adamw_step(th, g, m, v, t, lr, wd=0.01)
        binding.adamw_step(thd, torch.as_tensor(g, device="cuda"), md, vd, lr, t, weight_decay=0.01)
    torch.cuda.synchronize()
    np.testing.assert_allclose(thd.cpu().numpy(), th, rtol=1e-13, atol=1e-15)
    # the moments differ only by the rounding of fused multiply-adds
    np.testing.assert_allclose(md.cpu().numpy(), m, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(vd.cpu().numpy(), v, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("sampler", ["metropolis", "langevin"])
def test_training_lowers_the_h2_energy(lib, sampler):
    from paper_1909_08423_gb300.vmc import VMCTrainer
    sysd = synth.h2()
    s = lib.System(sysd, precision=lib.PN_MIXED, max_walkers=2048)
    tr = VMCTrainer(s, synth.flatten_params(sysd), walkers=512, batch=1024, resample_period=5, n_discard=50,
                    n_decorr=1, lr=0.01, t0=200, sampler=sampler, tau=0.1, seed=3)
    hist = [tr.step() for _ in range(100)]
    e = np.array([h["e_mean"] for h in hist])
    err = np.array([h["e_stderr"] for h in hist])
    assert np.all(np.isfinite(e))
    first, last = e[:5].mean(), e[-10:].mean()
    assert last < first - 0.02, (first, last)
    assert last > E_H2_EXACT - 5 * err[-10:].mean() - 0.01, (last, E_H2_EXACT)
