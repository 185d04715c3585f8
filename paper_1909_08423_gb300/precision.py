"""Per-system precision policy for the mixed path.

The tensor-core layers (tcgen05, three-piece bf16 operands, the leading
piece products accumulated apart from the others) are about as accurate as
CUDA-core float32, but how far the float32 network's rounding reaches the
local energy depends on the molecule (core electrons of heavy atoms and
walkers near nodes amplify it).  ``calibrate`` measures the local-energy
error of each tensor-core layer mask against the PN_FP64 path on walkers
sampled from |psi|^2 and returns the largest mask that keeps the stated
bounds.
"""

from __future__ import annotations

import torch

from . import binding

MASKS = (0, 4, 1 | 4, 2 | 4, 1 | 2 | 4)  # cheapest escalation last-to-first


def _eval(sysd, precision, mask, r, chunk):
    s = binding.System(sysd, precision=precision, max_walkers=chunk)
    if precision == binding.PN_MIXED:
        s.set_option(binding.PN_OPT_TENSOR_CORES, mask)
    E = torch.empty(r.shape[0], dtype=torch.float64, device=r.device)
    s.eval_local_energy(r, E)
    s.device_status()
    s.close()
    return E


def calibrate(sysd, r, max_err=1e-4, mean_err=1e-5, quantile=0.999, chunk=512):
    """r: sampled walkers on the device.  Returns (mask, table) where table
    maps each tried mask to (quantile error, mean error) in hartree."""
    ref = _eval(sysd, binding.PN_FP64, 0, r, chunk)
    table = {}
    best = 0
    for mask in MASKS:
        E = _eval(sysd, binding.PN_MIXED, mask, r, chunk)
        err = (E - ref).abs()
        q = float(torch.quantile(err, quantile))
        m = float(err.mean())
        table[mask] = (q, m)
        if q <= max_err and m <= mean_err:
            best = mask
    return best, table
