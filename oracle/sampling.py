"""Metropolis walker update and walker initialisation (Methods, "Ansatz
optimization": sampling from |psi|^2; the all-electron Gaussian proposal of
width sigma replaces the paper's Langevin proposal).  Test infrastructure only.

One step for every walker w:
  r' = r + sigma xi,  xi ~ N(0, 1) per coordinate (Philox stream, see philox)
  accept iff u < exp(2 (ln|psi(r')| - ln|psi(r)|)),  u ~ U(0, 1)
"""

from __future__ import annotations

import numpy as np

from paper_1909_08423_gb300 import synth

from . import philox


def metropolis(oracle, r, logabs, n_steps, sigma, seed, step0, walker0=0):
    r = np.array(r, dtype=np.float64)
    lp = np.array(logabs, dtype=np.float64)
    Wn, N, _ = r.shape
    walkers = np.arange(walker0, walker0 + Wn)
    n_acc = np.zeros(Wn, dtype=np.int64)
    for s in range(n_steps):
        step = step0 + s
        xi = philox.normals(seed, walkers, step, 3 * N).reshape(Wn, N, 3)
        u = philox.accept_uniform(seed, walkers, step, 3 * N)
        rn = r + sigma * xi
        lpn, _ = oracle.eval_logpsi(rn)
        acc = u < np.exp(2.0 * (lpn - lp))
        r = np.where(acc[:, None, None], rn, r)
        lp = np.where(acc, lpn, lp)
        n_acc += acc
    return r, lp, n_acc


def init_walkers(sys, W, seed, width=1.0):
    """Electron e at R[nucleus(e)] + width * normal, normals from the Philox
    stream at step 2^64 - 1 (normal index 3e + axis)."""
    nuc = synth.electron_nuclei(sys)
    N = len(nuc)
    xi = philox.normals(seed, np.arange(W), philox.INIT_STEP, 3 * N).reshape(W, N, 3)
    return sys["R"][nuc][None] + width * xi
