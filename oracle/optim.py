"""AdamW (Adam with decoupled weight decay, Loshchilov and Hutter), the
optimiser of the paper's ansatz optimisation (Methods), in plain numpy
float64.  Test infrastructure only.

For step t >= 1 with gradient g:
  m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2
  theta <- theta - lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps) + wd theta)
"""

from __future__ import annotations

import numpy as np


def adamw_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.01):
    """Returns the new (theta, m, v); the inputs are not modified."""
    m = b1 * np.asarray(m) + (1.0 - b1) * np.asarray(g)
    v = b2 * np.asarray(v) + (1.0 - b2) * np.asarray(g) ** 2
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    theta = np.asarray(theta) - lr * (mh / (np.sqrt(vh) + eps) + wd * np.asarray(theta))
    return theta, m, v


def learning_rate(t, lr0, t0):
    """Learning rate of training step t with decay period t0 (hyperparameter
    table): lr0 / (1 + t / t0)."""
    return lr0 / (1.0 + t / t0)
