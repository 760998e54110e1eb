"""Differentiable rollouts: a torch.autograd.Function whose forward is the library's
checkpointed time integration and whose backward is the library's reverse sweep.

The differentiable inputs are the parameters of the wetting walls, packed as one vector

    p = [dmu_w of cylinder 0 .. n_cyl-1, dmu_w of the flat walls, cx_0, cy_0, cx_1, cy_1, ...]

(the wall chemical-potential offsets of Eq. 15's boundary layer and the cylinder centres, which
enter the step through the cut fractions q of Eqs. 16-17), and the output is the fluid density
after n steps (ny x nx, zero off the fluid).  Any torch function of that density can be
differentiated back to p.
"""
from __future__ import annotations

import numpy as np

from . import _abi
from .lattice import Lattice


def params_vector(phys: dict) -> np.ndarray:
    """The parameter vector p of a physics dict."""
    n = len(phys.get("r", []))
    p = np.zeros(3 * n + 1)
    p[:n] = np.asarray(phys.get("dmu_w", []), np.float64)
    p[n] = float(phys.get("dmu_w_walls", 0.0))
    p[n + 1::2] = np.asarray(phys.get("cx", []), np.float64)
    p[n + 2::2] = np.asarray(phys.get("cy", []), np.float64)
    return p


def with_params(phys: dict, p) -> dict:
    """A copy of `phys` with the wall parameters taken from p."""
    n = len(phys.get("r", []))
    p = np.asarray(p, np.float64).reshape(-1)
    if p.size != 3 * n + 1:
        raise ValueError(f"parameter vector of length {p.size}, expected {3 * n + 1}")
    out = dict(phys)
    out["dmu_w"] = [float(v) for v in p[:n]]
    out["dmu_w_walls"] = float(p[n])
    out["cx"] = [float(v) for v in p[n + 1::2]]
    out["cy"] = [float(v) for v in p[n + 2::2]]
    return out


def _function():
    import torch

    class Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, phys, droplets, n_steps, every, precision):
            p = params.detach().to("cpu", torch.float64).numpy()
            lat = Lattice(with_params(phys, p), precision=precision)
            lat.init_droplets(droplets)
            lat.forward_checkpointed(int(n_steps), int(every))
            rho = lat.fields(on_device=True)[0]
            ctx.lat = lat
            ctx.pdtype, ctx.pdevice = params.dtype, params.device
            return rho

        @staticmethod
        def backward(ctx, g_rho):
            grad = ctx.lat.adjoint(drho=g_rho)
            g = torch.as_tensor(grad, dtype=ctx.pdtype, device=ctx.pdevice)
            return g, None, None, None, None, None

    return Rollout


_ROLLOUT = None


def rollout(params, phys: dict, droplets: dict, n_steps: int, every: int = 0, precision: int = _abi.LBM_FP32):
    """Fluid density after n_steps from the droplet initial state (Eq. 19), differentiable in
    the wall parameters `params` (a 1-D torch tensor, layout of params_vector)."""
    global _ROLLOUT
    if _ROLLOUT is None:
        _ROLLOUT = _function()
    return _ROLLOUT.apply(params, phys, droplets, n_steps, every, precision)
