"""torch.autograd.Function around lp_step / lp_step_adjoint.

Forward: nsteps FP64 LP steps whose stencils are rebuilt every
`checkpoint_every` steps and held fixed in between (the run the adjoint
differentiates). Backward: the hand-written adjoint gives dL/d(mu_s, mu_2, I0)
and dL/d(initial state) from dL/d(final state). Both run in the CUDA library;
this module only moves tensors.
"""
from __future__ import annotations

import torch

from . import capi

_MUI_REST = ("d", "rho_s")


class LPStepFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, x, y, z, u, v, w, V, ctx, mui_rest, eos, params, dt, nsteps,
                checkpoint_every):
        th = theta.detach().double().cpu().tolist()
        mui = dict(mu_s=th[0], mu_2=th[1], I0=th[2], **{k: mui_rest[k] for k in _MUI_REST})
        prm = dict(params, precision=capi.LP_FP64, rebuild_every=int(checkpoint_every),
                   launch_mode=capi.LP_LAUNCH_KERNELS)
        init = dict(x=x, y=y, z=z, u=u, v=v, w=w, V=V)
        st = {k: t.detach().clone().contiguous() for k, t in init.items()}
        capi.lp_step(ctx, st, mui, eos, prm, dt, int(nsteps))
        fctx.save_for_backward(*[init[k] for k in capi.FIELDS])
        fctx.meta = (ctx, mui, eos, prm, dt, int(nsteps), int(checkpoint_every), theta.device,
                     theta.dtype)
        return tuple(st[k] for k in capi.FIELDS)

    @staticmethod
    def backward(fctx, *grads):
        ctx, mui, eos, prm, dt, nsteps, cpe, tdev, tdt = fctx.meta
        init = dict(zip(capi.FIELDS, fctx.saved_tensors))
        seed = {k: (g.contiguous().double() if g is not None else torch.zeros_like(init[k]))
                for k, g in zip(capi.FIELDS, grads)}
        want_init = any(fctx.needs_input_grad[1:8])
        dmui, gi = capi.lp_step_adjoint(ctx, init, mui, eos, prm, dt, nsteps, cpe, seed,
                                        want_initial=want_init)
        gtheta = dmui.to(device=tdev, dtype=tdt)
        gstate = [gi[k] if gi is not None else None for k in capi.FIELDS]
        return (gtheta, *gstate) + (None,) * 7


def lp_step_diff(ctx, theta: torch.Tensor, state: dict, mui_rest: dict, eos: dict, params: dict,
                 dt: float, nsteps: int, checkpoint_every: int):
    """Differentiable LP run: returns the final state as a dict of tensors."""
    out = LPStepFunction.apply(theta, *[state[k] for k in capi.FIELDS], ctx, mui_rest, eos,
                               params, dt, nsteps, checkpoint_every)
    return dict(zip(capi.FIELDS, out))


def runout_profile_loss(state: dict, R: float, target: torch.Tensor, nbins: int = 32):
    """Runout max_i sqrt(x^2 + y^2) plus the squared misfit of the height
    profile (max z in nbins radial bins on [0, 3R]) to `target`. The argmax of
    each max is taken from the current values (ties to the lower index) and
    held fixed for the gradient."""
    x, y, z = state["x"], state["y"], state["z"]
    r = torch.sqrt(x * x + y * y)
    i_run = int(torch.argmax(r.detach()).item())
    runout = r[i_run]
    b = torch.clamp((r.detach() / (3.0 * R / nbins)).long(), 0, nbins - 1)
    zd = z.detach()
    idx = []
    for k in range(nbins):
        sel = torch.nonzero(b == k).flatten()
        idx.append(int(sel[torch.argmax(zd[sel])].item()) if sel.numel() else -1)
    heights = torch.stack([z[i] if i >= 0 else z.new_zeros(()) for i in idx])
    return runout + ((heights - target) ** 2).sum(), heights.detach()
