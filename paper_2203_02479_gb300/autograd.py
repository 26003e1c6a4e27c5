"""torch.autograd wrapper of the expected-value simulation and its adjoint.

``simulate(q, x_mm, t_us, DL, DT, R, plane, params)`` returns the simulated
grid M (nwires x nticks) through ``ws_simulate`` and differentiates it with
``ws_simulate_backward``: gradients flow to the depo charges, pitch
positions and drift times, to the diffusion constants D_L and D_T (0-dim
tensors) and to the response R.  Patches are recomputed in the backward
pass; only the three depo arrays and the response are saved.

A plane holds one response spectrum at a time.  Each forward records the R
it ran with, and each backward makes the plane hold that R again before the
adjoint runs, so several forwards on one plane (say a prediction and a
target under different responses) each get the gradients of their own R.
The spectrum is recomputed only when the plane holds another response than
the one a call needs (``Plane.use_response``).
"""
from __future__ import annotations

import dataclasses

import torch

from .wiresim import DeviceDepos, Params, Plane


class SimulateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, x, t, DL, DT, R, plane: Plane, params: Params):
        p = dataclasses.replace(params, DL_mm2_us=float(DL), DT_mm2_us=float(DT), fluctuate=False)
        Rd = R.detach()
        plane.use_response(Rd)
        depos = DeviceDepos(q.detach(), x.detach(), t.detach(), device=plane.device)
        M = plane.simulate(depos, p)
        ctx.save_for_backward(q, x, t, DL, DT, Rd)
        ctx.plane = plane
        ctx.params = p
        return M

    @staticmethod
    def backward(ctx, gM):
        q, x, t, DL, DT, R = ctx.saved_tensors
        plane = ctx.plane
        plane.use_response(R)      # the response this forward ran with
        depos = DeviceDepos(q.detach(), x.detach(), t.detach(), device=plane.device)
        gq, gx, gt, gDL, gDT, gR = plane.backward(depos, ctx.params, gM.detach().float().contiguous(),
                                                  want_response=ctx.needs_input_grad[5])
        gDL = gDL.to(DL.dtype).reshape(DL.shape)
        gDT = gDT.to(DT.dtype).reshape(DT.shape)
        return (gq.to(q.dtype), gx.to(x.dtype), gt.to(t.dtype), gDL, gDT,
                None if gR is None else gR, None, None)


def simulate(q, x_mm, t_us, DL, DT, R, plane: Plane, params: Params | None = None):
    """Differentiable expected-value simulation of one plane (see module doc)."""
    return SimulateFn.apply(q, x_mm, t_us, DL, DT, R, plane, params or Params())
