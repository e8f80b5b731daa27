"""torch.autograd wrapper of the micromagnetic energy (Eq. Hmm).

``EnergyFn.apply(m, L, disk_handle)`` returns the energy in joules of every
replica of a single-disk ``Nanodisk`` (FP64 field and sums in the library).
Its backward calls the library twice: ``nd_effective_field`` for
dE/dm_i = -J b_i (Eq. Bi: the effective induction is minus the energy
gradient in units of J, evaluated on the FFT path), and ``nd_energy`` with the
thickness derivative of the Green's tensor for dE/dL at fixed m.  The only
torch arithmetic is the chain-rule scaling of those library results by the
incoming gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from ._binding import nd_effective_field, nd_energy


def _replica_scale(h, values, device, dtype):
    """Per-element vector that holds values[r] on replica r's block."""
    s = torch.empty(h.state_elems, dtype=dtype, device=device)
    for r, L in enumerate(h.layout):
        n = 3 * L["D"] * L["Dpad"]
        s[L["offset"]:L["offset"] + n] = float(values[r])
    return s


class EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, L, h):
        assert len(h.disks) == 1, "EnergyFn expects a single-disk handle"
        Lv = float(L)
        assert abs(Lv - h.disks[0].L) <= 1e-12 * h.disks[0].L, "L must be the handle's disk thickness"
        E, dEdL = nd_energy(h.h, m, h.B, with_dL=True)
        J = h.units[0][4]
        ctx.save_for_backward(m)
        ctx.h, ctx.dEdL, ctx.J = h, dEdL, J
        return torch.as_tensor(E * J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gE):
        (m,) = ctx.saved_tensors
        h = ctx.h
        g = gE.detach().to("cpu", torch.float64).numpy()
        gm = gL = None
        if ctx.needs_input_grad[0]:
            b = torch.zeros_like(m)
            nd_effective_field(h.h, m, b)
            gm = b * _replica_scale(h, -ctx.J * g, m.device, m.dtype)
        if ctx.needs_input_grad[1]:
            gL = torch.as_tensor(float(np.dot(g, ctx.dEdL)), dtype=torch.float64)
        return gm, gL, None


def energy(m, L, h):
    """Energies in joules with autograd support for m and L."""
    return EnergyFn.apply(m, L, h)
