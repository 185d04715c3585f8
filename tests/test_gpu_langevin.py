"""Langevin (drift-diffusion) sampler through the C ABI against the oracle.

The drift grad ln|psi| of the FP64 path, formed both in reverse mode (the
default) and by the forward jet pass, matches the oracle's reverse-mode
gradient to rounding; the FP64 chain reproduces the oracle's chain (same
Philox stream, same clipping of the drift at the nearest nucleus); the
mixed chain makes only moves the oracle would propose from the same state,
with accept decisions that differ from the oracle's only at rounding-level
ties; and at full batch size the chain samples the hydrogen density.
"""

import numpy as np
import pytest
import torch

from oracle import philox, sampling
from oracle.ansatz import Oracle
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

SYSTEMS = {"be": synth.be, "h10": synth.h10, "n2": synth.n2}


@pytest.fixture(scope="module")
def oracles():
    return {k: Oracle(f()) for k, f in SYSTEMS.items()}


def _equilibrated(o, W, seed):
    r = synth.random_walkers(o.sys, W, seed)
    lp, _ = o.eval_logpsi(r)
    r, _, _ = sampling.metropolis(o, r, lp, 20, 0.2, seed=seed, step0=0)
    return r


@pytest.mark.parametrize("mode", [1, 0], ids=["reverse", "jet"])
@pytest.mark.parametrize("name,W", [("be", 64), ("h10", 16), ("n2", 6)])
def test_drift_matches_oracle(lib, oracles, name, W, mode):
    o = oracles[name]
    r = _equilibrated(o, W, 3)
    lp_o, _, g_o = o.value_and_grad(r)
    for prec, tol in ((0, 1e-8), (1, 2e-3)):
        s = lib.System(o.sys, precision=prec, max_walkers=32)
        s.set_option(lib.PN_OPT_DRIFT, mode)
        rd = torch.as_tensor(r, device="cuda")
        g = torch.empty_like(rd)
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        s.eval_drift(rd, g, lp)
        torch.cuda.synchronize()
        gn, lpn = g.cpu().numpy(), lp.cpu().numpy()
        scale = 1.0 + np.abs(g_o)
        if prec == 0:
            np.testing.assert_allclose(lpn, lp_o, rtol=0, atol=1e-9 * (1 + np.abs(lp_o)).max())
            assert np.max(np.abs(gn - g_o) / scale) < tol
        else:
            err = np.abs(gn - g_o) / scale
            assert np.median(err) < 1e-5 and np.max(err) < tol, (np.median(err), np.max(err))
        # host buffers give the same numbers
        gh = np.empty(r.shape)
        s.eval_drift(np.ascontiguousarray(r), gh)
        np.testing.assert_array_equal(gh, gn)


@pytest.mark.parametrize("mode", [1, 0], ids=["reverse", "jet"])
@pytest.mark.parametrize("name,W,steps,tau", [("be", 48, 4, 0.1), ("h10", 12, 2, 0.1), ("n2", 4, 2, 0.05)])
def test_langevin_fp64_matches_oracle(lib, oracles, name, W, steps, tau, mode):
    o = oracles[name]
    r0 = _equilibrated(o, W, 5)
    lp0, _, g0 = o.value_and_grad(r0)
    ro, lpo, go, acco = sampling.langevin(o, r0, lp0, g0, steps, tau, seed=11, step0=300)
    s = lib.System(o.sys, precision=lib.PN_FP64, max_walkers=32)
    s.set_option(lib.PN_OPT_DRIFT, mode)
    rd = torch.as_tensor(r0, device="cuda").clone()
    lpd = torch.as_tensor(lp0, device="cuda").clone()
    gd = torch.as_tensor(g0, device="cuda").clone()
    nacc = torch.zeros(1, dtype=torch.int64, device="cuda")
    s.langevin_step(rd, lpd, gd, steps, tau, 11, 300, nacc)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rd.cpu().numpy(), ro, rtol=0, atol=1e-9)
    np.testing.assert_allclose(lpd.cpu().numpy(), lpo, rtol=1e-11, atol=1e-10)
    np.testing.assert_allclose(gd.cpu().numpy(), go, rtol=1e-8, atol=1e-8)
    assert int(nacc.item()) == int(acco.sum())
    assert 0 < int(acco.sum()) < W * steps  # both outcomes occur


@pytest.mark.parametrize("name,W,steps", [("be", 64, 4), ("h10", 16, 2)])
def test_langevin_mixed_moves_are_valid(lib, oracles, name, W, steps):
    """From the mixed chain's own state each step: the walker stays or moves
    to r + c(r) + sqrt(tau) xi with c from the chain's drift; where its
    decision differs from the oracle's, the oracle's log ratio at that
    proposal lies within 1e-3 of ln u."""
    o = oracles[name]
    tau = 0.1
    N = o.N
    r0 = _equilibrated(o, W, 6)
    s = lib.System(o.sys, precision=lib.PN_MIXED, max_walkers=32)
    rd = torch.as_tensor(r0, device="cuda").clone()
    lpd = torch.empty(W, dtype=torch.float64, device="cuda")
    gd = torch.empty_like(rd)
    s.eval_drift(rd, gd, lpd)
    walkers = np.arange(W)
    flips = 0
    for k in range(steps):
        step = 700 + k
        r_old, g_old = rd.cpu().numpy(), gd.cpu().numpy()
        s.langevin_step(rd, lpd, gd, 1, tau, 13, step)
        torch.cuda.synchronize()
        r_new = rd.cpu().numpy()
        xi = philox.normals(13, walkers, step, 3 * N).reshape(W, N, 3)
        prop = r_old + sampling.clipped_drift(o.sys, r_old, g_old, tau) + np.sqrt(tau) * xi
        stay = np.all(r_new == r_old, axis=(1, 2))
        moved = np.all(np.abs(r_new - prop) < 1e-9, axis=(1, 2))
        assert np.all(stay | moved)
        lp_o, _, g_o = o.value_and_grad(r_old)
        lpp_o, _, gp_o = o.value_and_grad(prop)
        fwd = prop - r_old - sampling.clipped_drift(o.sys, r_old, g_o, tau)
        back = r_old - prop - sampling.clipped_drift(o.sys, prop, gp_o, tau)
        log_ratio = 2 * (lpp_o - lp_o) + ((fwd * fwd).sum((1, 2)) - (back * back).sum((1, 2))) / (2 * tau)
        u = philox.accept_uniform(13, walkers, step, 3 * N)
        margin = log_ratio - np.log(u)
        differ = moved != (margin > 0)
        assert np.all(np.abs(margin[differ]) < 1e-3), margin[differ]
        flips += int(differ.sum())
    assert flips <= max(1, W * steps // 20)


_VARIANTS = {
    # the ablation variants, a system without the cusp corrections and LiH
    "be_no_heads": lambda: synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=4, D=64, K=32, L=3,
                                             seed=0, no_jastrow=1, no_backflow=1),
    "be_no_backflow": lambda: synth.make_system([4.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=1, D=64, K=32, L=3,
                                                seed=0, no_backflow=1),
    "lih_plain": lambda: synth.lih(use_cusp=False, use_gamma=False),
    "lih": synth.lih,
}


@pytest.mark.parametrize("name", list(_VARIANTS))
def test_reverse_drift_equals_jet_drift(lib, name):
    """Both ways of forming grad_r ln|psi| give the same numbers: to rounding
    on the FP64 path, to float32 accuracy on the mixed path; chunked (W above
    the workspace) and host buffers included."""
    sysd = _VARIANTS[name]()
    W = 72
    r = synth.random_walkers(sysd, W, 8)
    for prec, tol in ((0, 1e-9), (1, 2e-3)):
        s = lib.System(sysd, precision=prec, max_walkers=32)
        out = {}
        for mode in (0, 1):
            s.set_option(lib.PN_OPT_DRIFT, mode)
            g = np.empty(r.shape)
            lp = np.empty(W)
            s.eval_drift(np.ascontiguousarray(r), g, lp)
            out[mode] = (g, lp)
        (g0, l0), (g1, l1) = out[0], out[1]
        fin = np.isfinite(l0)
        assert fin.mean() > 0.9
        np.testing.assert_array_equal(np.isfinite(l1), fin)
        np.testing.assert_allclose(l1[fin], l0[fin], rtol=0, atol=1e-10 if prec == 0 else 1e-4)
        err = np.abs(g1[fin] - g0[fin]) / (1.0 + np.abs(g0[fin]))
        assert err.max() < tol, (prec, err.max())


def test_drift_option_rejects_bad_values(lib):
    s = lib.System(synth.be(), precision=lib.PN_FP64, max_walkers=8)
    with pytest.raises(lib.PNError):
        s.set_option(lib.PN_OPT_DRIFT, 2)


@pytest.mark.parametrize("precision", [0, 1])
def test_langevin_samples_hydrogen_density_at_scale(lib, precision):
    """16384 walkers of the hydrogen atom (psi = exp(-r)): <r> = 3/2 and
    <r^2> = 3 after burn-in, acceptance high at tau = 0.1."""
    S = synth.hydrogen_like_sto(1.0, 1.0)
    s = lib.System(S, precision=precision, max_walkers=16384)
    W = 16384
    r = torch.empty(W, 1, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, 21)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    g = torch.empty_like(r)
    s.eval_drift(r, g, lp)
    s.langevin_step(r, lp, g, 60, 0.1, 21, 0)
    rs = []
    nacc = torch.zeros(1, dtype=torch.int64, device="cuda")
    for b in range(4):
        s.langevin_step(r, lp, g, 10, 0.1, 21, 60 + 10 * b, nacc)
        rs.append(torch.linalg.norm(r[:, 0], dim=-1).cpu().numpy())
    rs = np.concatenate(rs)
    assert abs(rs.mean() - 1.5) < 0.02
    assert abs((rs ** 2).mean() - 3.0) < 0.08
    assert int(nacc.item()) / (W * 10) > 0.95


def test_langevin_bad_arguments(lib):
    from paper_1909_08423_gb300 import binding
    S = synth.be()
    s = lib.System(S, precision=lib.PN_FP64, max_walkers=8)
    r = torch.zeros(4, 4, 3, dtype=torch.float64, device="cuda")
    lp = torch.zeros(4, dtype=torch.float64, device="cuda")
    g = torch.zeros_like(r)
    with pytest.raises(binding.PNError):
        s.langevin_step(r, lp, g, 1, 0.0, 1, 0)
    with pytest.raises(binding.PNError):
        s.langevin_step(r.cpu().numpy(), lp, g, 1, 0.1, 1, 0)
