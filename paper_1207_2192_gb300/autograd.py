"""torch.autograd wrappers of the micromagnetic energy and of the force
constant, and a constrained relaxation driven by the energy's gradient.

Equations are cited by the paper's own labels: Eq. Hmm is the effective 2D
Hamiltonian, Eq. Bi the local induction as minus its gradient, Eq. Ux the
parabolic energy of a displaced core that defines k_F.

``EnergyFn.apply(m, L, disk_handle)`` returns the energy in joules of every
replica of a single-disk ``Nanodisk`` (the energy of Eq. Hmm, Sec. II.A, with
an FP64 field and FP64 sums in the library).  Its backward calls the library
twice: ``nd_effective_field`` for dE/dm_i = -J b_i (the effective induction of
Eq. Bi is minus the energy gradient in units of J, evaluated on the FFT path)
and ``nd_energy`` with the thickness derivative of the Sec. II.B tensor for
dE/dL at fixed m.

``relax_by_energy_gradient`` runs the constrained relaxation of Sec. IV (the
sweep of ``nd_relax_constrained``) with the field taken from the gradient
that torch.autograd computes for the energy -- optionally plus energy terms
the caller writes in torch -- through ``nd_relax_sweep_grad``.

``ForceConstantFn.apply(aspect, radii, ...)`` returns the force constant k_F
(Eq. Ux: two constrained relaxations per disk, at X = 0 and X = 2a) of every
disk of a batch of any sizes as a function of the aspect ratios L/R at fixed
radii and masks; its backward is dk_F/d(L/R) = R dk_F/dL from the envelope
theorem (dU/dL at a constrained minimum is the partial derivative of the
energy at that state, which ``nd_energy`` returns).

The only torch arithmetic is the chain-rule scaling of library results by the
incoming gradients.
"""
from __future__ import annotations

import numpy as np
import torch

from ._binding import nd_effective_field, nd_energy, nd_relax_sweep_grad


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


def relax_by_energy_gradient(h, m, X, tol=1e-6, max_iter=20000, extra_energy=None):
    """Constrained relaxation of every replica of a single-disk handle with the
    core pinned at X ([B][2], metres), each sweep's field coming from the
    autograd gradient of E(m) = energy(m) (+ extra_energy(m), a torch scalar in
    joules the caller may add).  m (a device tensor) is updated in place.
    Returns dict(converged, lam [B][2], iters, resid [B])."""
    L = torch.tensor(h.disks[0].L, dtype=torch.float64)
    lam = np.zeros((h.B, 2))
    res = np.full(h.B, np.inf)
    for it in range(max_iter):
        mt = m.detach().requires_grad_(True)
        E = energy(mt, L, h).sum()
        if extra_energy is not None:
            E = E + extra_energy(mt)
        (g,) = torch.autograd.grad(E, mt)
        res, moved = nd_relax_sweep_grad(h.h, m, g, X, lam, h.B, tol)
        if not moved.any():
            return dict(converged=True, lam=lam, iters=it, resid=res)
    return dict(converged=False, lam=lam, iters=max_iter, resid=res)


class ForceConstantFn(torch.autograd.Function):
    """k_F of a batch of disks (radii fixed, any sizes: one batched relaxation
    over all their padded-size classes) as a differentiable function of the
    aspect ratios L/R."""

    @staticmethod
    def forward(ctx, aspect, radii, a, tol, precision):
        from .physics import geometry_sweep
        Rs = [float(R) for R in radii]
        asp = aspect.detach().to("cpu", torch.float64).numpy()
        res = geometry_sweep(Rs, [float(x) * R for x, R in zip(asp, Rs)], a=a, tol=tol, precision=precision)
        ctx.save_for_backward(torch.tensor([R * r["dkF_dL"] for R, r in zip(Rs, res)], dtype=torch.float64))
        ctx.converged = [r["converged"] for r in res]
        return torch.tensor([r["kF"] for r in res], dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        (dk,) = ctx.saved_tensors
        return g.to(torch.float64) * dk, None, None, None, None


def force_constants(aspect, radii, a=2e-9, tol=1e-6, precision=None):
    """k_F (N/m) of disks of radii R and aspect ratios L/R (a tensor that may
    require grad): backward gives dk_F/d(L/R)."""
    return ForceConstantFn.apply(aspect, radii, a, tol, precision)
