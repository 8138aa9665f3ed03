"""Time-averaged lift and drag as differentiable functions of the airfoil
shape and incidence, for PyTorch optimisers.

`mean_force(case, amplitudes, aoa_deg, n_steps, wd, wl, skip=0)` returns J =
mean over coarse steps skip .. n_steps - 1 of wd C_D + wl C_L for the geometry
with the thickness bumps t(x) += A_m sin(m pi x) (workloads.thickness_modes)
and the given angle of attack, as a torch scalar whose backward pass is the
library's discrete adjoint (hlbm_adjoint): dJ/dA_m = dJ/dx . (mode m field),
dJ/d(angle) directly.  Each call builds an FP64 solver for the moved geometry
on the current CUDA device and runs the adjoint once (forward value and
gradients together).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def _moved_case(case, amplitudes, aoa_deg, modes):
    xy = case.xy + np.tensordot(np.asarray(amplitudes, dtype=np.float64), modes, axes=1)
    return dataclasses.replace(case, xy=xy, aoa_deg=float(aoa_deg))


def mean_force(case, amplitudes, aoa_deg, n_steps=10, wd=1.0, wl=0.0, modes=None, skip=0):
    """J(amplitudes [M], aoa_deg []) as a differentiable torch scalar (FP64):
    the mean over coarse steps skip .. n_steps - 1."""
    import torch

    from . import Solver
    from workloads import thickness_modes

    if modes is None:
        modes = thickness_modes(case, int(amplitudes.numel()))

    class _MeanForce(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a, alpha):
            moved = _moved_case(case, a.detach().cpu().numpy(), float(alpha.detach().cpu()), modes)
            sol = Solver(moved, precision="fp64")
            J, _, _, gx, da = sol.adjoint(int(n_steps), float(wd), float(wl), int(skip))
            sol.close()
            dA = np.array([float((gx * f).sum()) for f in modes])
            ctx.save_for_backward(torch.as_tensor(dA, dtype=a.dtype, device=a.device),
                                  torch.as_tensor(da, dtype=alpha.dtype, device=alpha.device))
            return torch.as_tensor(J, dtype=torch.float64, device=a.device)

        @staticmethod
        def backward(ctx, grad_out):
            dA, da = ctx.saved_tensors
            return grad_out * dA, grad_out * da

    return _MeanForce.apply(amplitudes, aoa_deg)
