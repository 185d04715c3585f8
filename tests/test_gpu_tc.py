"""Tensor-core (tcgen05) linear layer against a float64 product.

Operands are split into three bf16 pieces and six piece products are
accumulated in float32, which must keep float32-level accuracy: the error is
held to 2^-20 of sum_k |x_k w_k| per element, the size of float32 rounding
of a K-term sum (measured worst case 3.6e-7, i.e. 2^-21.4)."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [(1, 8, 16, 1), (127, 32, 32, 14), (128, 64, 32, 1), (300, 96, 64, 14), (5000, 64, 6, 14),
          (1000, 192, 128, 1), (257, 40, 1, 5), (4096, 64, 256, 14)]


@pytest.mark.parametrize("rows,K,Nout,T", SHAPES)
@pytest.mark.parametrize("acc", [0, 1])
def test_tc_linear_matches_float64(lib, rows, K, Nout, T, acc):
    cdll = lib.load()
    g = torch.Generator().manual_seed(rows * 31 + K)
    X = torch.randn(rows, K, generator=g, dtype=torch.float64)
    W = torch.randn(K, Nout, generator=g, dtype=torch.float64) * 0.1
    b = torch.randn(Nout, generator=g, dtype=torch.float64)
    Y0 = torch.randn(rows, Nout, generator=g, dtype=torch.float64)
    Xf, Wf, bf = X.float(), W.float(), b.float()
    ref = Xf.double() @ Wf.double()
    val = (torch.arange(rows) % T == 0).double()[:, None]
    ref = ref + val * bf.double()[None, :]
    Yd = Y0.float().cuda()
    if acc:
        ref = ref + Y0.float().double()
    Xd, Wd, bd = Xf.cuda(), Wf.cuda(), bf.cuda()
    rc = cdll.pn_test_linear_tc(Xd.data_ptr(), K, Wd.data_ptr(), Nout, bd.data_ptr(), Yd.data_ptr(), Nout, rows, K,
                                Nout, T, acc, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, cdll.pn_last_error()
    scale = (Xf.double().abs() @ Wf.double().abs()) + val * bf.double().abs()[None, :] + (Y0.abs() if acc else 0)
    err = (Yd.cpu().double() - ref).abs()
    assert torch.all(err <= 2.0 ** -20 * scale + 1e-30), float((err / scale).max())
