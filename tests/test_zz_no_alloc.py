"""The allocation-free value pass, pn_eval_logpsi_static.

It exists for callers that may not allocate device memory while they
evaluate (for example a latency-bound loop that must not wait on the
allocator, or a service that reserves its memory once at start-up): the call
keeps its intermediates in a fixed device array instead of allocating.  Its
results must equal those of pn_eval_logpsi, call after call, since the fixed
array is reused, and a call must leave the device's free memory as it found
it.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1909_08423_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_fn(lib):
    cdll = lib.load()
    f = cdll.pn_eval_logpsi_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return cdll, f


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_matches_allocating_entry_point(lib, precision):
    cdll, f = _static_fn(lib)
    sysd = synth.be()
    s = lib.System(sysd, precision=precision, max_walkers=256)
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((41, 42)):
        W = 300 + 17 * call
        r = torch.as_tensor(synth.random_walkers(sysd, W, seed), device="cuda")
        ref_lp = torch.empty(W, dtype=torch.float64, device="cuda")
        ref_sg = torch.empty_like(ref_lp)
        s.eval_logpsi(r, ref_lp, ref_sg)
        lp = torch.full((W,), np.nan, dtype=torch.float64, device="cuda")
        sg = torch.full((W,), np.nan, dtype=torch.float64, device="cuda")
        st = torch.full((W,), -1, dtype=torch.int32, device="cuda")
        rc = f(s.h, r.data_ptr(), W, lp.data_ptr(), sg.data_ptr(), st.data_ptr(), stream)
        assert rc == 0, cdll.pn_last_error()
        torch.cuda.synchronize()
        a, b = lp.cpu().numpy(), ref_lp.cpu().numpy()
        assert np.all(np.abs(a - b) <= 1e-9 * (1 + np.abs(b)))
        np.testing.assert_array_equal(sg.cpu().numpy(), ref_sg.cpu().numpy())
        assert np.all(st.cpu().numpy() == 0)


def test_static_call_leaves_free_device_memory_unchanged(lib):
    cdll, f = _static_fn(lib)
    sysd = synth.be()
    s = lib.System(sysd, precision=1, max_walkers=64)
    W = 256
    r = torch.as_tensor(synth.random_walkers(sysd, W, 43), device="cuda")
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert f(s.h, r.data_ptr(), W, lp.data_ptr(), None, None, stream) == 0  # first call: symbol lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert f(s.h, r.data_ptr(), W, lp.data_ptr(), None, None, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_rejects_oversized_batches(lib):
    cdll, f = _static_fn(lib)
    sysd = synth.be()
    s = lib.System(sysd, precision=0, max_walkers=64)
    W = 100000
    r = torch.zeros(W, s.N, 3, dtype=torch.float64, device="cuda")
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    rc = f(s.h, r.data_ptr(), W, lp.data_ptr(), None, None, torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert b"static scratch holds" in cdll.pn_last_error()
