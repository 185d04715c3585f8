"""Metropolis walker updates and walker initialisation (Methods, "Ansatz
optimization": sampling from |psi|^2): the all-electron Gaussian proposal of
width sigma, and the paper's Langevin (drift-diffusion) proposal with the
step-length clipping at the nearest nucleus.  Test infrastructure only.

Gaussian proposal, one step for every walker w:
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


def clipped_drift(sys, r, grad, tau):
    """Drift displacement of the Langevin proposal: c_i = tau grad_i ln|psi|,
    shortened to the distance from electron i to its nearest nucleus when it
    is longer, so that the drift cannot carry an electron past a nucleus
    (Methods, sampling: the step-length clipping that replaces the radial
    proposal of Umrigar et al.)."""
    d = np.linalg.norm(r[:, :, None, :] - np.asarray(sys["R"])[None, None], axis=-1).min(-1)  # [W,N]
    c = tau * grad
    length = np.linalg.norm(c, axis=-1)
    scale = np.where(length > d, d / np.where(length > 0, length, 1.0), 1.0)
    return c * scale[..., None]


def langevin(oracle, r, logabs, grad, n_steps, tau, seed, step0, walker0=0):
    """Langevin (drift-diffusion) Metropolis-Hastings steps for all walkers:
      r' = r + c(r) + sqrt(tau) xi,  c = clipped_drift,  xi ~ N(0, 1) (Philox)
      accept iff u < |psi(r')/psi(r)|^2 T(r' -> r) / T(r -> r'),
      T(x -> y) = exp(-|y - x - c(x)|^2 / (2 tau)).
    The normals and the uniform come from the same Philox stream layout as
    `metropolis`.  Returns r, ln|psi|, grad ln|psi| and the accept counts."""
    sys = oracle.sys
    r = np.array(r, dtype=np.float64)
    lp = np.array(logabs, dtype=np.float64)
    g = np.array(grad, dtype=np.float64)
    Wn, N, _ = r.shape
    walkers = np.arange(walker0, walker0 + Wn)
    n_acc = np.zeros(Wn, dtype=np.int64)
    for s in range(n_steps):
        step = step0 + s
        xi = philox.normals(seed, walkers, step, 3 * N).reshape(Wn, N, 3)
        u = philox.accept_uniform(seed, walkers, step, 3 * N)
        rn = r + clipped_drift(sys, r, g, tau) + np.sqrt(tau) * xi
        lpn, _, gn = oracle.value_and_grad(rn)
        back = r - rn - clipped_drift(sys, rn, gn, tau)
        log_ratio = 2.0 * (lpn - lp) + 0.5 * (xi * xi).sum((1, 2)) - (back * back).sum((1, 2)) / (2.0 * tau)
        acc = u < np.exp(log_ratio)
        r = np.where(acc[:, None, None], rn, r)
        lp = np.where(acc, lpn, lp)
        g = np.where(acc[:, None, None], gn, g)
        n_acc += acc
    return r, lp, g, n_acc


def init_walkers(sys, W, seed, width=1.0):
    """Electron e at R[nucleus(e)] + width * normal, normals from the Philox
    stream at step 2^64 - 1 (normal index 3e + axis)."""
    nuc = synth.electron_nuclei(sys)
    N = len(nuc)
    xi = philox.normals(seed, np.arange(W), philox.INIT_STEP, 3 * N).reshape(W, N, 3)
    return sys["R"][nuc][None] + width * xi
