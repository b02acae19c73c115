"""torch.autograd wrapper of the pathwise adjoint (``xy_adjoint_step_n``)."""
from __future__ import annotations

import torch


class BBKObjective(torch.autograd.Function):
    """objective = (1/(B n)) sum_b sum_{k=k0+1}^{k0+n} [w_E E_k + w_M |M_k|]
    over n BBK steps from the lattice's current state (which advances by n),
    with the noise held fixed.  Inputs J_par, J_perp, h, eta: tensors of shape
    (n_cfg,) (one value per configuration); their gradients come from the
    library's reverse sweep."""

    @staticmethod
    def forward(ctx, J_par, J_perp, h, eta, lattice, n, checkpoint_every, w_E, w_M):
        for c in range(len(lattice.configs)):
            prm = dict(lattice.configs[c].params)
            prm.update(J_par=float(J_par[c]), J_perp=float(J_perp[c]), h=float(h[c]), eta=float(eta[c]))
            lattice.set_params(c, **prm)
        obj, grads = lattice.adjoint(n, checkpoint_every, w_E, w_M)
        g = torch.as_tensor(grads, dtype=J_par.dtype, device=J_par.device)
        ctx.save_for_backward(g)
        return torch.tensor(obj, dtype=J_par.dtype, device=J_par.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return (grad_out * g[:, 0], grad_out * g[:, 1], grad_out * g[:, 2], grad_out * g[:, 3],
                None, None, None, None, None)


def bbk_objective(lattice, J_par, J_perp, h, eta, n, checkpoint_every=100, w_E=1.0, w_M=0.0):
    return BBKObjective.apply(J_par, J_perp, h, eta, lattice, n, checkpoint_every, w_E, w_M)
