"""The determinant jet by the table method (PN_OPT_DET_TABLE 1, the
default) against the block-by-block kernel (0) and the table kernel's own
block-by-block fallback (2), in float64 where the three must agree to
rounding amplified by the conditioning of determinant 0's blocks."""

import numpy as np
import pytest
import torch

from oracle.ansatz import Oracle
from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu

SYSTEMS = {"be": synth.be, "h10": synth.h10, "n2": synth.n2, "lih": synth.lih,
           "serve7": lambda: synth.serving_system(7)}


def _eval(lib, sysd, r, mode, chunk=512):
    s = lib.System(sysd, precision=lib.PN_FP64, max_walkers=chunk)
    s.set_option(lib.PN_OPT_DET_TABLE, mode)
    s.set_option(lib.PN_OPT_DRIFT, 0)  # drift from the jet pass: the determinants' gradients
    W = r.shape[0]
    E = torch.empty(W, dtype=torch.float64, device="cuda")
    lp = torch.empty_like(E)
    sg = torch.empty_like(E)
    st = torch.empty(W, dtype=torch.int32, device="cuda")
    s.eval_local_energy(r, E, lp, sg, st)
    g = torch.empty_like(r)
    s.eval_drift(r, g)
    torch.cuda.synchronize()
    return E.cpu().numpy(), lp.cpu().numpy(), sg.cpu().numpy(), st.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_table_matches_block_by_block(lib, name):
    sysd = SYSTEMS[name]()
    W = 1500
    r = torch.as_tensor(synth.random_walkers(sysd, W, 21), device="cuda")
    out = {m: _eval(lib, sysd, r, m) for m in (0, 1, 2)}
    E0, lp0, sg0, st0, g0 = out[0]
    ok = st0 == 0
    for m in (1, 2):
        E, lp, sg, st, g = out[m]
        np.testing.assert_array_equal(st, st0)
        np.testing.assert_array_equal(sg[ok], sg0[ok])
        np.testing.assert_allclose(lp[ok], lp0[ok], rtol=1e-11, atol=1e-10)
        assert np.all(np.abs(E[ok] - E0[ok]) <= 1e-8 * (1 + np.abs(E0[ok]))), np.max(np.abs(E[ok] - E0[ok]))
        scale = 1 + np.abs(g0[ok]).max(axis=(1, 2), keepdims=True)
        assert np.all(np.abs(g[ok] - g0[ok]) <= 1e-8 * scale)


def test_table_matches_oracle_on_n2(lib):
    """The default path against the oracle (float64) on 16 N2-shaped walkers."""
    sysd = synth.n2()
    r = synth.random_walkers(sysd, 16, 22)
    E, lp, _, st, _ = _eval(lib, sysd, torch.as_tensor(r, device="cuda"), 1)
    Eo, lpo, _ = Oracle(sysd).local_energy(r)
    assert np.all(st == 0)
    assert np.all(np.abs(E - Eo) <= 1e-8 * (1 + np.abs(Eo)))
    np.testing.assert_allclose(lp, lpo, rtol=1e-11, atol=1e-10)
