"""The MAHI energy as a differentiable torch function.

``MahiEnergy`` holds a solver handle for a fixed system layout (box, site map,
order, depth, precision).  ``energy(x, lam, qA, qB)`` returns the HI energy as
a 0-d tensor whose backward pass is one library kernel (``mahi_backward``):
dE/dx = -F, dE/dlambda, dE/dqA and dE/dqB come from the forward evaluation's
forces, lambda-derivatives and potentials (Eqs. "DeltaFQIHI", "Udiff" with
q~ = (1 - lambda) qA + lambda qB).  Argument marshalling only: nothing here
computes on the host.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Mahi, mahi_backward


class _Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, lam, qA, qB, owner):
        owner._sync_charges(qA, qB, x.device)
        E, F, g = owner.solver.eval(x.contiguous(), lam.contiguous())
        owner._evals += 1
        ctx.owner = owner
        ctx.eval_id = owner._evals
        ctx.save_for_backward(F, g, lam)
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE):
        owner = ctx.owner
        if owner._evals != ctx.eval_id:
            raise RuntimeError("MahiEnergy: another evaluation ran on this solver since this forward pass; "
                               "the backward pass needs the potentials of its own forward pass")
        F, g, lam = ctx.saved_tensors
        need = ctx.needs_input_grad
        dev = F.device
        n = owner.solver.n_atoms
        dx = torch.empty_like(F) if need[0] else None
        dl = torch.empty_like(g) if need[1] else None
        dqA = torch.empty(n, dtype=torch.float64, device=dev) if need[2] else None
        dqB = torch.empty(n, dtype=torch.float64, device=dev) if need[3] else None
        ge = gE.detach().to(dtype=torch.float64, device=dev).reshape(1).contiguous()
        mahi_backward(owner.solver.h, ge, F, g, lam, dx, dl, dqA, dqB)
        return dx, dl, dqA, dqB, None


class MahiEnergy:
    """Differentiable HI energy of a fixed system layout.

    site_of: host int array (-1 = environment, else the site index); charges are
    passed per call (device tensors of n_atoms float64).  The first call hands
    them to mahi_set_charges (which validates the site map); later changes go
    through mahi_update_charges, a device-side copy enqueued on the solver's
    stream (no host round trip).  Environment atoms must have qA == qB; their
    gradient goes to qA."""

    def __init__(self, box_L_nm, site_of, n_sites, order_p, depth, precision="mixed", stream=None):
        self.site_of = np.ascontiguousarray(site_of, dtype=np.int32)
        self.solver = Mahi(box_L_nm, len(self.site_of), n_sites, order_p, depth, precision, stream)
        self._key = None
        self._keep = None
        self._evals = 0

    def _sync_charges(self, qA, qB, device):
        key = (qA.data_ptr(), qA._version, qB.data_ptr(), qB._version)
        if key != self._key:
            a = qA.detach().to(device=device, dtype=torch.float64).contiguous()
            b = qB.detach().to(device=device, dtype=torch.float64).contiguous()
            if self._key is None:
                self.solver.set_charges(a, b, self.site_of)
            else:
                self.solver.update_charges(a, b)
            self._keep = (a, b)   # alive until the stream has read them
            self._key = key

    def energy(self, x, lam, qA, qB):
        return _Fn.apply(x, lam, qA, qB, self)

    def close(self):
        self.solver.close()
