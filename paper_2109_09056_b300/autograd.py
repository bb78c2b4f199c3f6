"""torch.autograd.Function for force matching: forward = md_compute_forces,
backward = md_force_backward (the hand-written FP64 adjoint kernel).

    F, E = LJForce.apply(x, eps, sigma, system)

x: (n, 3) float64 positions; eps, sigma: (ntypes, ntypes) float64 symmetric
tables; system: an MDSystem whose types and box define the rest.  F is the
(n, 3) FP64 force tensor and E the potential energy (0-d tensor).  The
backward re-bins, re-sorts and rebuilds the neighbor list from the saved
positions; no list is kept from the forward pass.
"""
from __future__ import annotations

import numpy as np
import torch

from .api import MDSystem


class LJForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, eps, sigma, system: MDSystem):
        system.set_params(eps.detach().cpu().numpy(), sigma.detach().cpu().numpy())
        system.set_positions(x.detach())
        energy = system.compute_forces()
        st = system.state(device=x.device)
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
        dx, de, ds = system.force_backward(gF, ge, device=x.device)
        if not isinstance(dx, torch.Tensor):
            dx = torch.from_numpy(np.asarray(dx))
        return (dx.to(x.device), torch.from_numpy(de).to(eps.device),
                torch.from_numpy(ds).to(sigma.device), None)
