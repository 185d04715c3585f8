"""Ablation variants of the ansatz (Results: single vs multiple determinants,
with and without backflow; and both heads removed), through the C ABI
against the oracle, which implements them by their definition (J = 0,
f = 1)."""

import numpy as np
import pytest
import torch

from oracle import sampling
from oracle.ansatz import Oracle
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

VARIANTS = {
    # name: (n_det, no_jastrow, no_backflow)
    "SD-SJ": (1, 0, 1),
    "SD-BF": (1, 0, 0),
    "MD-SJ": (4, 0, 1),
    "MD-BF": (4, 0, 0),
    "MD-none": (4, 1, 1),
}


def _be(variant):
    nd, nj, nb = VARIANTS[variant]
    return synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=nd, D=64, K=32, L=3, seed=0,
                             no_jastrow=nj, no_backflow=nb)


def _head_ranges(sysd):
    sh = synth.param_shapes(sysd["D"], sysd["Zd"], sysd["K"], sysd["L"], len(sysd["Z"]), sysd["mo_coeffs"].shape[1])
    out, off = {}, 0
    for name, shape in sh:
        n = int(np.prod(shape))
        head = name.split(".")[0]
        if head in ("eta", "kappa"):
            a, b = out.get(head, (off, off))
            out[head] = (min(a, off), off + n)
        off += n
    return out


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_variant_fp64_matches_oracle(lib, variant):
    sysd = _be(variant)
    o = Oracle(sysd)
    r = synth.random_walkers(sysd, 40, 3)
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=32)
    rd = torch.as_tensor(r, device="cuda")
    E = torch.empty(40, dtype=torch.float64, device="cuda")
    lp = torch.empty_like(E)
    s.eval_local_energy(rd, E, lp)
    torch.cuda.synchronize()
    Eo, lpo, _ = o.local_energy(r)
    ok = np.abs(Eo) < 1e4  # walkers away from nodes
    np.testing.assert_allclose(E.cpu().numpy()[ok], Eo[ok], rtol=0, atol=1e-8 * (1 + np.abs(Eo[ok])).max())
    np.testing.assert_allclose(lp.cpu().numpy(), lpo, rtol=1e-11, atol=1e-10)
    cot = torch.as_tensor(np.random.default_rng(4).normal(size=40), device="cuda")
    g = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
    s.grad_logpsi(rd, cot, g)
    torch.cuda.synchronize()
    gn = g.cpu().numpy()
    go = o.grad_logpsi(r, cot.cpu().numpy())
    np.testing.assert_allclose(gn, go, rtol=1e-9, atol=1e-11 * max(1.0, np.abs(go).max()))
    nd, nj, nb = VARIANTS[variant]
    heads = _head_ranges(sysd)
    if nj:
        a, b = heads["eta"]
        assert np.all(gn[a:b] == 0)
    if nb:
        a, b = heads["kappa"]
        assert np.all(gn[a:b] == 0)


@pytest.mark.parametrize("variant", ["SD-SJ", "MD-SJ"])
def test_variant_mixed_sampler_follows_the_oracle(lib, variant):
    """The tensor-core sampler on a variant without backflow: at least 90 % of
    the chains equal the oracle's after 6 steps (the rest differ only by
    rounding-level accept ties)."""
    sysd = _be(variant)
    o = Oracle(sysd)
    W = 96
    r0 = synth.random_walkers(sysd, W, 9)
    lp0, _ = o.eval_logpsi(r0)
    ro, _, _ = sampling.metropolis(o, r0, lp0, 6, 0.2, seed=77, step0=1000)
    s = lib.System(sysd, precision=lib.PN_MIXED, max_walkers=W)
    rd = torch.as_tensor(r0, device="cuda").clone()
    lpd = torch.as_tensor(lp0, device="cuda").clone()
    s.metropolis_step(rd, lpd, 6, 0.2, 77, 1000)
    torch.cuda.synchronize()
    same = np.all(np.abs(rd.cpu().numpy() - ro) < 1e-5, axis=(1, 2))
    assert same.mean() > 0.9


def test_set_params_keeps_the_variant(lib):
    """New parameters do not bring a removed head back."""
    sysd = _be("MD-SJ")
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=8)
    flat = synth.flatten_params(sysd)
    rng = np.random.default_rng(5)
    new = flat + rng.normal(0, 0.05, flat.shape)
    s.set_params(new)
    sys2 = dict(sysd)
    sys2["params"] = synth.unflatten_params(sysd, new)
    o2 = Oracle(sys2)
    r = synth.random_walkers(sysd, 8, 2)
    lp = torch.empty(8, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    s.eval_logpsi(torch.as_tensor(r, device="cuda"), lp, sg)
    torch.cuda.synchronize()
    lpo, _ = o2.eval_logpsi(r)
    np.testing.assert_allclose(lp.cpu().numpy(), lpo, rtol=1e-11, atol=1e-10)
