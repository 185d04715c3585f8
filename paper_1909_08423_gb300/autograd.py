"""torch.autograd.Function around the library's hand-written backward.

``LogPsi.apply(params, r, system)`` returns ln|psi(r)| per walker; its
backward calls pn_grad_logpsi with the incoming per-walker cotangent, so
``(weights * logpsi).sum().backward()`` yields sum_w weights_w grad ln|psi_w|,
the quantity Eq. (trainig) of the paper needs.  ``vmc_loss_and_grad``
assembles the whole VMC loss gradient on the device: local energies,
clipping, per-walker weights 2 (E_w - L) / W, backward.
"""

from __future__ import annotations

import torch

from . import binding


class LogPsi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, r, system):
        system.set_params(params.detach().contiguous())
        lp = torch.empty(r.shape[0], dtype=torch.float64, device=r.device)
        sg = torch.empty_like(lp)
        system.eval_logpsi(r, lp, sg)
        ctx.save_for_backward(r)
        ctx.system = system
        ctx.n_params = params.numel()
        return lp

    @staticmethod
    def backward(ctx, g):
        (r,) = ctx.saved_tensors
        grad = torch.empty(ctx.n_params, dtype=torch.float64, device=r.device)
        ctx.system.grad_logpsi(r, g.detach().contiguous().to(torch.float64), grad)
        return grad, None, None


def vmc_loss_and_grad(system, r, q=5.0, mem_budget_bytes=0, clip_fn=None, group=None):
    """Clipped mean local energy L and grad_theta L = sum_w u_w grad ln|psi_w|
    with u_w = 2 (E'_w - L) / W (E' the clipped local energies).

    Under torch.distributed with more than one rank, r holds this rank's
    walkers and the exchange steps run over `group`: the clipping window is
    taken over every rank's local energies, W is the total walker count, and
    the gradient is summed over ranks, so every rank returns the loss and
    gradient of the whole batch.  clip_fn(E, E_clipped, cot) defaults to the
    library's clipping kernel."""
    from . import distributed as pd
    clip_fn = clip_fn or (lambda E, Ec, cot: binding.clip_local_energy(E, Ec, cot, q))
    W = r.shape[0]
    E = torch.empty(W, dtype=torch.float64, device=r.device)
    system.eval_local_energy(r, E)
    grad = torch.empty(system.n_params, dtype=torch.float64, device=r.device)
    if pd.world_size(group) > 1:
        Ec, cot, loss = pd.global_clip(E, clip_fn, group)
        system.grad_logpsi(r, cot, grad, mem_budget_bytes)
        pd.allreduce_grad(grad, group)
        return loss, grad, E
    Ec = torch.empty_like(E)
    cot = torch.empty_like(E)
    clip_fn(E, Ec, cot)
    system.grad_logpsi(r, cot, grad, mem_budget_bytes)
    return Ec.mean(), grad, E
