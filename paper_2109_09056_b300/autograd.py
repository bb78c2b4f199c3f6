"""torch.autograd.Function for force matching: forward = md_compute_forces,
backward = md_force_backward (the hand-written FP64 adjoint kernel).

    F, E = LJForce.apply(x, eps, sigma, system)

x: (n, 3) float64 positions; eps, sigma: (ntypes, ntypes) float64 symmetric
tables; system: an MDSystem whose types and box define the rest.  F is the
(n, 3) FP64 force tensor and E the potential energy (0-d tensor).  The
backward re-bins, re-sorts and rebuilds the neighbor list from the saved
positions; no list is kept from the forward pass.

Gradient convention for the tables: md_force_backward returns, for an
unordered type pair {a, b}, the derivative with respect to the one parameter
both entries hold.  autograd treats eps[a, b] and eps[b, a] as two entries,
so each off-diagonal entry receives half of it; for any symmetric
parameterisation (eps = (E + E^T) / 2, a shared scalar, ...) the chain rule
then gives the exact gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from .api import MDSystem


def _entrywise(g: np.ndarray) -> np.ndarray:
    out = 0.5 * g
    np.fill_diagonal(out, np.diag(g))
    return out


class LJForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, eps, sigma, system: MDSystem):
        system.set_params(eps.detach().cpu().numpy(), sigma.detach().cpu().numpy())
        system.set_positions(x.detach())
        energy = system.compute_forces()
        st = system.state(device=x.device if x.is_cuda else None)
        ctx.system = system
        ctx.save_for_backward(x.detach(), eps.detach(), sigma.detach())
        f = st["f"]
        if not isinstance(f, torch.Tensor):
            f = torch.from_numpy(f)
        return f.to(x.device), torch.tensor(energy, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, gF, gE):
        x, eps, sigma = ctx.saved_tensors
        system = ctx.system
        system.set_params(eps.cpu().numpy(), sigma.cpu().numpy())
        system.set_positions(x)
        gF = torch.zeros_like(x) if gF is None else gF.contiguous().to(torch.float64)
        ge = 0.0 if gE is None else float(gE)
        dx, de, ds = system.force_backward(gF, ge, device=x.device if x.is_cuda else None)
        if not isinstance(dx, torch.Tensor):
            dx = torch.from_numpy(np.asarray(dx))
        return (dx.to(x.device), torch.from_numpy(_entrywise(de)).to(eps.device),
                torch.from_numpy(_entrywise(ds)).to(sigma.device), None)
