"""Hand-written backward of ln|psi| (pn_grad_logpsi) against the oracle's
reverse mode and against central differences of the GPU's own ln|psi|."""

import numpy as np
import pytest
import torch

from oracle.ansatz import Oracle
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,W", [(synth.h2, 40), (synth.be, 50), (synth.h10, 20), (synth.n2, 6)])
def test_grad_fp64_matches_oracle(lib, make, W):
    sysd = make()
    r = synth.random_walkers(sysd, W, 21)
    cot = np.random.default_rng(2).normal(size=W)
    g_or = Oracle(sysd).grad_logpsi(r, cot)
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=64)
    g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
    s.grad_logpsi(torch.as_tensor(r, device="cuda"), torch.as_tensor(cot, device="cuda"), g)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    scale = np.abs(g_or).max()
    np.testing.assert_allclose(g, g_or, rtol=1e-9, atol=1e-11 * scale)


def test_grad_chunking_by_memory_budget(lib):
    sysd = synth.be()
    r = torch.as_tensor(synth.random_walkers(sysd, 300, 3), device="cuda")
    cot = torch.as_tensor(np.random.default_rng(0).normal(size=300), device="cuda")
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=512)
    outs = []
    for budget in (0, 30 << 20, 16 << 20):
        g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
        s.grad_logpsi(r, cot, g, budget)
        outs.append(g.cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_allclose(o, outs[0], rtol=1e-11, atol=1e-13 * np.abs(outs[0]).max())


def test_grad_matches_finite_differences_h10(lib):
    """Central differences of the GPU's ln|psi| on 64 seeded parameters."""
    sysd = synth.h10()
    W = 16
    r = torch.as_tensor(synth.random_walkers(sysd, W, 4), device="cuda")
    cot = torch.as_tensor(np.random.default_rng(1).normal(size=W), device="cuda")
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=W)
    g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
    s.grad_logpsi(r, cot, g)
    g = g.cpu().numpy()
    flat = synth.flatten_params(sysd)
    idx = np.random.default_rng(64).choice(len(flat), 64, replace=False)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    h = 1e-5
    for k in idx:
        vals = []
        for sgn in (1, -1):
            fl = flat.copy()
            fl[k] += sgn * h
            s.set_params(fl)
            s.eval_logpsi(r, lp, sg)
            vals.append(float((lp * cot).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
    s.set_params(flat)


def test_grad_mixed_close_to_fp64(lib):
    sysd = synth.h10()
    r = torch.as_tensor(synth.random_walkers(sysd, 64, 5), device="cuda")
    cot = torch.as_tensor(np.random.default_rng(3).normal(size=64), device="cuda")
    g = {}
    for p in (lib.PN_FP64, lib.PN_MIXED):
        s = lib.System(sysd, precision=p, max_walkers=64)
        out = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
        s.grad_logpsi(r, cot, out)
        g[p] = out.cpu().numpy()
    # element by element: within 1e-3 of the entry plus 1e-5 of the largest
    # entry (the float32 network's accumulated rounding, with a margin)
    bound = 1e-3 * np.abs(g[0]) + 1e-5 * np.abs(g[0]).max()
    assert np.all(np.abs(g[1] - g[0]) <= bound), np.max(np.abs(g[1] - g[0]) / bound)


def test_autograd_function_and_vmc_gradient(lib):
    from paper_1909_08423_gb300.autograd import LogPsi, vmc_loss_and_grad
    from oracle import clip as oclip
    sysd = synth.be()
    W = 64
    rn = synth.random_walkers(sysd, W, 6)
    r = torch.as_tensor(rn, device="cuda")
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=W)
    params = torch.as_tensor(synth.flatten_params(sysd), device="cuda").requires_grad_(True)
    w = torch.as_tensor(np.random.default_rng(9).normal(size=W), device="cuda")
    (LogPsi.apply(params, r, s) * w).sum().backward()
    o = Oracle(sysd)
    np.testing.assert_allclose(params.grad.cpu().numpy(), o.grad_logpsi(rn, w.cpu().numpy()), rtol=1e-9,
                               atol=1e-11)
    L, grad, E = vmc_loss_and_grad(s, r)
    Eo, _, _ = o.local_energy(rn)
    Ec = oclip.clip_local_energy(Eo)
    ref = o.grad_logpsi(rn, oclip.loss_cotangent(Ec))
    np.testing.assert_allclose(float(L), Ec.mean(), rtol=1e-10)
    np.testing.assert_allclose(grad.cpu().numpy(), ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
