"""Edges of the C ABI: empty batches, a single walker, systems at every
compiled maximum (32 electrons with 16 per spin, 32 orbitals, 64
determinants, 8 interaction layers, D = 256; 16 nuclei), and descriptions
one step beyond a maximum, which init rejects with a message."""

import numpy as np
import pytest
import torch

from oracle import sampling
from oracle.ansatz import Oracle
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu


def _max_system():
    """Four Z=8 nuclei on a 2.8-bohr square: 32 electrons (16 per spin), 36
    basis functions, 32 orbitals, 64 determinants, D = 256, 8 layers.  The
    seeded weights are scaled by 0.3 so that eight layers of width 256 keep
    ln|psi| near its orbital part instead of growing to 1e6."""
    R = [[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0], [2.8, 2.8, 0]]
    s = synth.make_system([8.0] * 4, R, lambda z: {0: 3, 1: 2}, n_det=64, D=256, K=32, L=8, seed=4, n_orb=32)
    s["params"] = {k: np.asarray(v) * 0.3 for k, v in s["params"].items()}
    return s


def _sixteen_nuclei():
    R = [[1.8 * (i % 4), 1.8 * (i // 4), 0.0] for i in range(16)]
    return synth.make_system([1.0] * 16, R, lambda z: {0: 3}, n_det=4, D=64, K=32, L=2, seed=5)


def test_empty_batches_do_nothing(lib):
    sysd = synth.be()
    for prec in (lib.PN_FP64, lib.PN_MIXED):
        s = lib.System(sysd, precision=prec, max_walkers=16)
        r = torch.empty(0, s.N, 3, dtype=torch.float64, device="cuda")
        v = torch.empty(0, dtype=torch.float64, device="cuda")
        s.eval_logpsi(r, v, v)
        s.eval_local_energy(r, v)
        nacc = torch.full((1,), 7, dtype=torch.int64, device="cuda")
        s.metropolis_step(r, v, 5, 0.2, 1, 0, nacc)
        torch.cuda.synchronize()
        assert int(nacc.item()) == 0
        s.init_walkers(r, 1)
        s.eval_drift(r, r, v)
        s.langevin_step(r, v, r, 3, 0.1, 1, 0)
        g = torch.full((s.n_params,), np.nan, dtype=torch.float64, device="cuda")
        s.grad_logpsi(r, v, g)
        torch.cuda.synchronize()
        assert torch.all(g == 0)


def test_single_walker_matches_oracle(lib):
    sysd = synth.be()
    o = Oracle(sysd)
    r = synth.random_walkers(sysd, 1, 4)
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=1)
    rd = torch.as_tensor(r, device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    lp = torch.empty_like(E)
    s.eval_local_energy(rd, E, lp)
    torch.cuda.synchronize()
    Eo, lpo, _ = o.local_energy(r)
    np.testing.assert_allclose(E.cpu().numpy(), Eo, rtol=1e-9)
    np.testing.assert_allclose(lp.cpu().numpy(), lpo, rtol=1e-11)
    ro, lpr, _ = sampling.metropolis(o, r, lpo, 4, 0.2, seed=9, step0=0)
    s.metropolis_step(rd, lp, 4, 0.2, 9, 0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rd.cpu().numpy(), ro, rtol=0, atol=1e-10)


def test_system_at_every_maximum(lib):
    sysd = _max_system()
    o = Oracle(sysd)
    W = 4
    r = synth.random_walkers(sysd, W, 1)
    lpo, sgo = o.eval_logpsi(r)
    for prec, tol in ((lib.PN_FP64, 1e-10), (lib.PN_MIXED, 1e-5)):
        s = lib.System(sysd, precision=prec, max_walkers=W)
        assert s.N == 32
        rd = torch.as_tensor(r, device="cuda")
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(lp)
        s.eval_logpsi(rd, lp, sg)
        torch.cuda.synchronize()
        np.testing.assert_allclose(lp.cpu().numpy(), lpo, rtol=tol)
        np.testing.assert_array_equal(sg.cpu().numpy(), sgo)
        if prec == lib.PN_FP64:
            E = torch.empty(1, dtype=torch.float64, device="cuda")
            s.eval_local_energy(rd[:1].contiguous(), E)
            torch.cuda.synchronize()
            Eo, _, _ = o.local_energy(r[:1])
            np.testing.assert_allclose(E.cpu().numpy(), Eo, rtol=1e-8)
            ro, _, _ = sampling.metropolis(o, r, lpo, 2, 0.1, seed=2, step0=0)
            lpd = torch.as_tensor(lpo, device="cuda").clone()
            s.metropolis_step(rd, lpd, 2, 0.1, 2, 0)
            torch.cuda.synchronize()
            np.testing.assert_allclose(rd.cpu().numpy(), ro, rtol=0, atol=1e-9)


def test_sixteen_nuclei(lib):
    sysd = _sixteen_nuclei()
    o = Oracle(sysd)
    r = synth.random_walkers(sysd, 2, 2)
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=2)
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    s.eval_local_energy(torch.as_tensor(r, device="cuda"), E)
    torch.cuda.synchronize()
    Eo, _, _ = o.local_energy(r)
    np.testing.assert_allclose(E.cpu().numpy(), Eo, rtol=1e-8)


@pytest.mark.parametrize("what", ["electrons", "dets", "layers", "dim", "nuclei"])
def test_descriptions_beyond_a_maximum_are_rejected(lib, what):
    from paper_1909_08423_gb300 import binding
    if what == "electrons":  # 33 electrons
        sysd = synth.make_system([8.0] * 4 + [1.0], [[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0], [2.8, 2.8, 0], [5, 5, 5]],
                                 lambda z: {0: 3, 1: 2}, n_det=1, D=32, K=16, L=1, seed=1)
    elif what == "dets":
        sysd = synth.make_system([8.0] * 4, [[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0], [2.8, 2.8, 0]],
                                 lambda z: {0: 3, 1: 2}, n_det=65, D=32, K=16, L=1, seed=1, n_orb=32)
    elif what == "layers":
        sysd = synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=1, D=32, K=16, L=9, seed=1)
    elif what == "dim":
        sysd = synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=1, D=272, K=16, L=1, seed=1)
    else:  # 17 nuclei
        sysd = synth.make_system([1.0] * 17, [[1.8 * i, 0, 0] for i in range(17)], lambda z: {0: 3}, n_det=1, D=32,
                                 K=16, L=1, seed=1)
    with pytest.raises(binding.PNError) as e:
        binding.System(sysd)
    assert e.value.code == 1
    assert "outside" in str(e.value) or "range" in str(e.value), str(e.value)


@pytest.mark.parametrize("fused", [4, 1])
def test_one_electron_sampler_density(lib, fused):
    """The mixed samplers (tensor-core and warp kernels) on the hydrogen atom,
    one electron and no electron pairs: 16384 walkers reproduce the moments
    <r> = 3/2 and <r^2> = 3 of |psi|^2 = exp(-2r)."""
    S = synth.hydrogen_like_sto(1.0, 1.0)
    s = lib.System(S, precision=lib.PN_MIXED, max_walkers=16384)
    s.set_option(lib.PN_OPT_FUSED_SAMPLER, fused)
    W = 16384
    r = torch.empty(W, 1, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, 5)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    s.eval_logpsi(r, lp, sg)
    s.metropolis_step(r, lp, 100, 0.5, 5, 0)
    rs = []
    for b in range(4):
        s.metropolis_step(r, lp, 10, 0.5, 5, 100 + 10 * b)
        rs.append(torch.linalg.norm(r[:, 0], dim=-1).cpu().numpy())
    rs = np.concatenate(rs)
    assert abs(rs.mean() - 1.5) < 0.02
    assert abs((rs ** 2).mean() - 3.0) < 0.08
