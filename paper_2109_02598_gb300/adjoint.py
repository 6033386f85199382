"""Gradients of a final-state loss through the forward-Euler time loop (2D grids).

``GrayScottAdjoint`` and ``PhaseFieldAdjoint`` are ``torch.autograd.Function`` wrappers over
the library's adjoint entry points (``pf_adj_forward`` / ``pf_adj_backward`` in
include/pfgpu.h): the forward pass advances the initial fields by n steps with sqrt(N)
checkpointing, the backward pass runs the hand-written adjoint kernels and returns the
gradient with respect to the initial fields and the model coefficients -- Gray-Scott
(Du, Dv, F, k), Model A (c1, c2), Model B (c1, c2, mobility M).  Argument marshalling only;
all arithmetic runs in libpfgpu's kernels.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import check
from .grid import Grid, _torch


def adjoint_forward(grid: Grid, n_steps: int, ckpt_interval: int = 0):
    """pf_adj_forward on ``grid`` (Gray-Scott model and fields already set)."""
    check(grid._lib.pf_adj_forward(grid.handle, int(n_steps), int(ckpt_interval)))


def adjoint_backward(grid: Grid, dLdu_N, dLdv_N=None):
    """pf_adj_backward with CUDA tensors.

    Returns (dL/dx0 of field 0, of field 1 or None, [dL/dcoeff, ...]) with the coefficients
    in ``set_model`` order.
    """
    torch = _torch()
    gu = dLdu_N.detach().to(torch.float32).contiguous()
    du0 = torch.empty_like(gu)
    gv = dv0 = None
    if grid.n_fields == 2:
        gv = dLdv_N.detach().to(torch.float32).contiguous()
        dv0 = torch.empty_like(gv)
    dth = (ctypes.c_double * 4)()
    check(grid._lib.pf_adj_backward(grid.handle, ctypes.c_void_p(gu.data_ptr()),
                                    ctypes.c_void_p(gv.data_ptr() if gv is not None else None), 1,
                                    ctypes.c_void_p(du0.data_ptr()),
                                    ctypes.c_void_p(dv0.data_ptr() if dv0 is not None else None),
                                    dth))
    return du0, dv0, list(dth)[:len(grid.coeffs)]


class GrayScottAdjoint:
    """``apply(u0, v0, theta, n_steps, dt, h=1.0, ckpt_interval=0) -> (u_N, v_N)``.

    ``u0``, ``v0``: CUDA float32 tensors (ny, nx); ``theta``: tensor (Du, Dv, F, k).
    Gradients flow to u0, v0 and theta.
    """

    _fn = None

    @classmethod
    def _function(cls):
        if cls._fn is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, u0, v0, theta, n_steps, dt, h, ckpt_interval):
                    grid = Grid(tuple(u0.shape), 2, h)
                    grid.set_model("gs", [float(t) for t in theta.detach().cpu().tolist()], dt)
                    grid.write_field(0, u0)
                    grid.write_field(1, v0)
                    adjoint_forward(grid, n_steps, ckpt_interval)
                    uN = grid.read_field(0, device=True)
                    vN = grid.read_field(1, device=True)
                    grid.synchronize()
                    ctx.grid = grid
                    ctx.theta_meta = (theta.dtype, theta.device)
                    return uN, vN

                @staticmethod
                def backward(ctx, gu, gv):
                    torch = _torch()
                    grid = ctx.grid
                    if gu is None:
                        gu = torch.zeros(grid.shape, device="cuda")
                    if gv is None:
                        gv = torch.zeros(grid.shape, device="cuda")
                    du0, dv0, dth = adjoint_backward(grid, gu, gv)
                    dtype, device = ctx.theta_meta
                    grid.close()
                    ctx.grid = None
                    return (du0, dv0, torch.tensor(dth, dtype=dtype, device=device),
                            None, None, None, None)

            cls._fn = _Fn
        return cls._fn

    @classmethod
    def apply(cls, u0, v0, theta, n_steps: int, dt: float, h: float = 1.0,
              ckpt_interval: int = 0):
        return cls._function().apply(u0, v0, theta, int(n_steps), float(dt), float(h),
                                     int(ckpt_interval))


class PhaseFieldAdjoint:
    """``apply(phi0, theta, model, n_steps, dt, h=1.0, ckpt_interval=0) -> phi_N`` for
    Model A (``"ac"``, theta = (c1, c2)) or Model B (``"ch"``, theta = (c1, c2, M)).

    Gradients flow to phi0 and theta (including the mobility M of Model B).
    """

    _fn = None

    @classmethod
    def _function(cls):
        if cls._fn is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, phi0, theta, model, n_steps, dt, h, ckpt_interval):
                    grid = Grid(tuple(phi0.shape), 1, h)
                    grid.set_model(model, [float(t) for t in theta.detach().cpu().tolist()], dt)
                    grid.write_field(0, phi0)
                    adjoint_forward(grid, n_steps, ckpt_interval)
                    out = grid.read_field(0, device=True)
                    grid.synchronize()
                    ctx.grid = grid
                    ctx.theta_meta = (theta.dtype, theta.device)
                    return out

                @staticmethod
                def backward(ctx, g):
                    torch = _torch()
                    grid = ctx.grid
                    d0, _, dth = adjoint_backward(grid, g)
                    dtype, device = ctx.theta_meta
                    grid.close()
                    ctx.grid = None
                    return (d0, torch.tensor(dth, dtype=dtype, device=device),
                            None, None, None, None, None)

            cls._fn = _Fn
        return cls._fn

    @classmethod
    def apply(cls, phi0, theta, model: str, n_steps: int, dt: float, h: float = 1.0,
              ckpt_interval: int = 0):
        if model not in ("ac", "ch"):
            raise ValueError("PhaseFieldAdjoint takes model 'ac' or 'ch'")
        return cls._function().apply(phi0, theta, model, int(n_steps), float(dt), float(h),
                                     int(ckpt_interval))
