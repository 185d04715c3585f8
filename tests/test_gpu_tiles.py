"""Float32 tile kernels at widths the workload systems do not reach.

A carbon-like atom (6 electrons, 21 pairs per walker) with filter width 128
(eight 16-column groups per filter tile, 128 x 128 GEMM tiles for the
width-128 maps) and one with ragged widths (filter width 40, K = 24) run
the mixed path against the FP64 path on the same walkers; the FP64 path
uses the per-row kernels that the oracle tests pin.  The jet filter tiles
start at 128 k pair rows, so the local-energy case uses 8192 walkers in one
workspace chunk.
"""

import numpy as np
import pytest
import torch

from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = {"wide": dict(D=128, Zd=128, K=64), "ragged": dict(D=64, Zd=40, K=24)}


def _system(kind):
    return synth.make_system([6.0], [[0, 0, 0]], lambda z: {0: 4, 1: 2}, n_det=2, L=2, seed=3, **DIMS[kind])


def _equilibrated(lib, sysd, W, seed):
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=W)
    r = torch.empty(W, s.N, 3, dtype=torch.float64, device="cuda")
    s.init_walkers(r, seed)
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(lp)
    s.eval_logpsi(r, lp, sg)
    s.metropolis_step(r, lp, 30, 0.2, seed, 0)
    torch.cuda.synchronize()
    s.close()
    return r


@pytest.mark.parametrize("kind", list(DIMS))
def test_jet_tiles_local_energy(lib, kind):
    sysd = _system(kind)
    W = 8192
    r = _equilibrated(lib, sysd, W, 4)
    out = {}
    for prec in (lib.PN_FP64, lib.PN_MIXED):
        s = lib.System(sysd, precision=prec, max_walkers=W)
        E = torch.empty(W, dtype=torch.float64, device="cuda")
        lp = torch.empty_like(E)
        s.eval_local_energy(r, E, lp)
        torch.cuda.synchronize()
        out[prec] = (E.cpu().numpy(), lp.cpu().numpy())
        s.close()
    (E64, l64), (E32, l32) = out[lib.PN_FP64], out[lib.PN_MIXED]
    fin = np.isfinite(E64) & np.isfinite(l64)
    assert fin.mean() > 0.99
    np.testing.assert_array_equal(np.isfinite(E32[fin]), True)
    np.testing.assert_allclose(l32[fin], l64[fin], rtol=0, atol=1e-4)
    rel = np.abs(E32[fin] - E64[fin]) / (1.0 + np.abs(E64[fin]))
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-3, (np.median(rel), np.quantile(rel, 0.99))


@pytest.mark.parametrize("kind", list(DIMS))
def test_value_and_backward_tiles_gradient(lib, kind):
    sysd = _system(kind)
    W = 64
    r = _equilibrated(lib, sysd, W, 5)
    cot = torch.as_tensor(np.random.default_rng(6).normal(size=W), device="cuda")
    g = {}
    for prec in (lib.PN_FP64, lib.PN_MIXED):
        s = lib.System(sysd, precision=prec, max_walkers=W)
        out = torch.empty(s.n_params, dtype=torch.float64, device="cuda")
        s.grad_logpsi(r, cot, out)
        torch.cuda.synchronize()
        g[prec] = out.cpu().numpy()
        s.close()
    rel = np.linalg.norm(g[lib.PN_MIXED] - g[lib.PN_FP64]) / np.linalg.norm(g[lib.PN_FP64])
    assert rel < 1e-4, rel


@pytest.mark.parametrize("kind", list(DIMS))
def test_distance_tiles_drift(lib, kind):
    sysd = _system(kind)
    W = 64
    r = _equilibrated(lib, sysd, W, 7)
    d = {}
    for prec in (lib.PN_FP64, lib.PN_MIXED):
        s = lib.System(sysd, precision=prec, max_walkers=W)
        g = torch.empty_like(r)
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        s.eval_drift(r, g, lp)
        torch.cuda.synchronize()
        d[prec] = (g.cpu().numpy(), lp.cpu().numpy())
        s.close()
    (g64, l64), (g32, l32) = d[lib.PN_FP64], d[lib.PN_MIXED]
    np.testing.assert_allclose(l32, l64, rtol=0, atol=1e-4)
    err = np.abs(g32 - g64) / (1.0 + np.abs(g64))
    assert np.median(err) < 1e-5 and err.max() < 2e-3, (np.median(err), err.max())
