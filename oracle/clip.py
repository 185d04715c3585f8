"""Smooth clipping of local energies (Methods, "Ansatz optimization"): outside
a window of q times the mean absolute deviation from the batch median, values
grow only logarithmically.  Test infrastructure only.

  m = median(E) (mean of the two middle values for even counts),
  d = mean |E - m|,  L = q d
  E' = E                                   if |E - m| <= L
  E' = m + sgn(E - m) L (1 + ln(|E - m| / L))   otherwise
The map is continuous with a continuous first derivative at |E - m| = L.
"""

from __future__ import annotations

import numpy as np


def clip_local_energy(E, q=5.0):
    E = np.asarray(E, dtype=np.float64)
    m = np.median(E)
    d = np.mean(np.abs(E - m))
    L = q * d
    dev = E - m
    out = E.copy()
    big = np.abs(dev) > L
    out[big] = m + np.sign(dev[big]) * L * (1.0 + np.log(np.abs(dev[big]) / L))
    return out


def loss_cotangent(E_clipped):
    """Per-walker weights u_w = 2 (E_w - L) / W with L = mean(E): the VMC loss
    gradient of Eq. (trainig) is sum_w u_w grad_theta ln|psi_w|."""
    E = np.asarray(E_clipped, dtype=np.float64)
    return 2.0 * (E - E.mean()) / len(E)
