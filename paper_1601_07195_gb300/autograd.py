"""PyTorch autograd front end of the adjoint gradient.

``AdjointEnergy`` makes the energies E_i(theta) = <psi_i|H_i|psi_i> of a batch
of variational instances (``qs.Batch``) a differentiable function of one 1-D
float64 tensor holding every instance's angles, concatenated in instance order.
Its forward pass is one ``qs_batch_execute``: the adjoint reverse sweep
(Jones & Gacon, arXiv:2009.02823) yields the energies and every dE_i/dtheta in
the same launch sequence on the GPU, so the forward keeps the gradient vector
(one double per angle, the size of the angles themselves) and the backward
pass only scales it by the incoming gradient of each instance's energy:
d(loss)/d(theta_p) = d(loss)/d(E_i) * dE_i/d(theta_p) for the instance i that
owns angle p.  No second sweep runs in backward.

Only argument marshalling happens here; the circuits run in libqs.so.
"""

import numpy as np
import torch

from . import qs


class AdjointEnergy(torch.autograd.Function):
    """energies = AdjointEnergy.apply(theta, batch).

    theta: 1-D float64 tensor (any device) with sum(batch.sizes) angles.
    batch: a ``qs.Batch`` (its circuits and observables are fixed; its angles
    are replaced by theta at every call).
    Returns the instances' energies as a float64 tensor on theta's device.
    Second derivatives are not provided (backward is not differentiable).
    """

    @staticmethod
    def forward(ctx, theta, batch):
        if theta.dim() != 1 or theta.numel() != sum(batch.sizes):
            raise ValueError(f"theta must be 1-D with {sum(batch.sizes)} angles")
        th = theta.detach().to("cpu", torch.float64).numpy()
        thetas = np.split(th, np.cumsum(batch.sizes)[:-1]) if len(batch.sizes) > 1 else [th]
        energies, grads = batch.execute(thetas)
        g = np.concatenate(grads) if grads else np.zeros(0)
        ctx.save_for_backward(torch.from_numpy(g).to(theta.device))
        ctx.owner = torch.from_numpy(np.repeat(np.arange(len(batch.sizes)), batch.sizes)).to(theta.device)
        return torch.from_numpy(energies).to(theta.device)

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, grad_energies):
        (grads,) = ctx.saved_tensors
        return grad_energies.to(grads.dtype)[ctx.owner] * grads, None


def energies(batch, theta):
    """Differentiable energies of ``batch`` at the concatenated angles ``theta``."""
    return AdjointEnergy.apply(theta, batch)


def make_batch(instances, dtype=qs.QS_C128, stream=None):
    """A ``qs.Batch`` for use with ``energies`` (see qs.Batch for the instance records)."""
    return qs.Batch(instances, dtype, stream=stream)
