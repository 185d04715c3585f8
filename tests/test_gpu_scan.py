"""Line scans of E_loc through coalescences (Results, the one-dimensional
scan of the wave function and its local energy in LiH), through the C ABI
and through the serving loop."""

import numpy as np
import pytest
import torch

from oracle.ansatz import Oracle
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

NPTS = 256


def _scan(lib, sysd, precision, t0=None, t1=None, npts=NPTS, max_walkers=64):
    r0, e, d, a, b = synth.lih_scan()
    t0 = a if t0 is None else t0
    t1 = b if t1 is None else t1
    s = lib.System(sysd, precision=precision, max_walkers=max_walkers)
    E = torch.empty(npts, dtype=torch.float64, device="cuda")
    lp = torch.empty_like(E)
    s.eval_line_scan(torch.as_tensor(r0, device="cuda"), e, d, t0, t1, npts, E, lp)
    torch.cuda.synchronize()
    return E.cpu().numpy(), lp.cpu().numpy()


def _points(t0, t1, npts):
    r0, e, d, _, _ = synth.lih_scan()
    ts = t0 + np.arange(npts) * ((t1 - t0) / (npts - 1) if npts > 1 else 0.0)
    r = np.repeat(r0[None], npts, 0).copy()
    r[:, e, :] = r0[e] + ts[:, None] * d
    return r, ts


@pytest.mark.parametrize("chunk", [64, 1000])
def test_scan_matches_oracle(lib, chunk):
    sysd = synth.lih()
    o = Oracle(sysd)
    _, _, _, t0, t1 = synth.lih_scan()
    E, lp = _scan(lib, sysd, lib.PN_FP64, max_walkers=chunk)
    r, ts = _points(t0, t1, NPTS)
    idx = np.linspace(0, NPTS - 1, 16).astype(int)
    Eo, lpo, _ = o.local_energy(r[idx])
    np.testing.assert_allclose(E[idx], Eo, rtol=0, atol=1e-8 * (1 + np.abs(Eo)).max())
    np.testing.assert_allclose(lp[idx], lpo, rtol=1e-11, atol=1e-10)
    # the mixed path along the whole line, away from the same-spin node at
    # x = 1 (where psi vanishes and the determinant is ill conditioned)
    Em, _ = _scan(lib, sysd, lib.PN_MIXED, max_walkers=chunk)
    away = np.abs(ts - 1.0) > 0.1
    assert np.all(np.abs(Em[away] - E[away]) < 1e-3 * (1 + np.abs(E[away])))


@pytest.mark.parametrize("precision", [0, 1])
def test_scan_shows_the_cusps(lib, precision):
    """E_loc converges at the Li nucleus and at the opposite-spin electron
    with the cusp splice and gamma; without the splice it diverges like -Z/d
    at the nucleus, without gamma like +1/d at the electron."""
    deltas = [1e-2, 1e-3, 1e-4]

    def at(sysd, centre, side):
        return np.array([_scan(lib, sysd, precision, centre + side * dl, centre + side * dl, 1)[0][0] for dl in deltas])

    on = synth.lih()
    for centre in (0.0, 2.0):
        for side in (1.0, -1.0):
            E = at(on, centre, side)
            assert np.all(np.isfinite(E))
            assert abs(E[2] - E[1]) < abs(E[1] - E[0]) + 1e-6
            assert abs(E[2] - E[1]) < 0.1 * max(1.0, abs(E[1]))
    E = at(synth.lih(use_cusp=0), 0.0, 1.0)
    assert abs(E[2] * deltas[2] + 3.0) < 0.01
    E = at(synth.lih(use_gamma=0), 2.0, 1.0)
    assert abs(E[2] * deltas[2] - 1.0) < 0.01


def test_scan_job_through_the_server(lib):
    sysd = synth.lih()
    r0, e, d, t0, t1 = synth.lih_scan()
    E, _ = _scan(lib, sysd, lib.PN_MIXED, max_walkers=128)
    s = lib.System(sysd, precision=lib.PN_MIXED, max_walkers=1)
    srv = lib.Server(4 << 30, n_slots=2, chunk_walkers=128)
    out = torch.full((NPTS,), np.nan, dtype=torch.float64, device="cuda")
    jid = srv.submit(s, lib.PN_JOB_SCAN, NPTS, r_init=torch.as_tensor(r0, device="cuda"), eloc_out=out,
                     scan_electron=e, scan_dir=d, scan_t0=t0, scan_t1=t1)
    res = srv.poll(jid, timeout_us=-1)
    torch.cuda.synchronize()
    assert res.status == 0 and res.W == NPTS
    np.testing.assert_array_equal(out.cpu().numpy(), E)
    fin = np.isfinite(E)
    assert abs(res.e_mean - E[fin].mean()) < 1e-9 * max(1.0, abs(E[fin].mean()))
    srv.close()
