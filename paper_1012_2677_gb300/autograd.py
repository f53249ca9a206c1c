"""Differentiable velocity-Verlet trajectory as a torch.autograd.Function.

``LJTrajectory.apply(x0, v0, eps, sigma, box, dt, nsteps, n_pe, ckpt_every)`` returns the loss
  loss = (1 / n_pe) sum over the last n_pe states of PE / N  +  (1 / N) sum_i |x_i(n) - x_i(0)|^2
of an NVE run of the truncated LJ system (Eq. 2, r_c = rc_over_sigma * sigma).  Its gradients
with respect to x0, v0, eps and sigma come from the library's reverse-time pass through
velocity-Verlet (Hessian-vector products of the adjoint kernel, checkpoints every ckpt_every
steps).  When any input needs a gradient, the one library call that computes the loss also
runs the reverse pass, and backward() scales the stored gradients by the incoming one.
Marshalling only: all arithmetic runs in libljmd's kernels.
"""
from __future__ import annotations

import torch

from . import ljmd


class LJTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, eps, sigma, box, dt, nsteps, n_pe, ckpt_every, rc_over_sigma=2.5, margin=0.5,
                precision=ljmd.LJ_MIXED):
        if not (x0.is_cuda and v0.is_cuda):
            raise ValueError("x0 and v0 must be CUDA tensors")
        x0c = x0.detach().to(torch.float64).contiguous()
        v0c = v0.detach().to(torch.float64).contiguous()
        n = x0c.numel() // 3
        e, sg = float(eps), float(sigma)
        want = any(ctx.needs_input_grad[:4])
        gx = torch.empty_like(x0c) if want else None
        gv = torch.empty_like(v0c) if want else None
        with ljmd.System(eps=e, sigma=sg, cutoff=rc_over_sigma * sg, margin=margin, precision=precision,
                         energy_every=0, stream=torch.cuda.current_stream(x0.device)) as s:
            loss, gth = ljmd.ljmd_traj_loss_grad(s.h, n, float(box), x0c, v0c, float(dt), int(nsteps), int(n_pe),
                                                 int(ckpt_every), gx, gv)
        if want:
            dev = x0.device
            ctx.save_for_backward(gx.view_as(x0), gv.view_as(v0),
                                  torch.tensor(gth[0], dtype=torch.float64, device=dev),
                                  torch.tensor(gth[1], dtype=torch.float64, device=dev))
        return torch.tensor(loss, dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(ctx, g):
        gx, gv, ge, gs = ctx.saved_tensors
        return (g * gx, g * gv, (g * ge).to(torch.float64), (g * gs).to(torch.float64),
                None, None, None, None, None, None, None, None)


def trajectory_loss(x0, v0, eps, sigma, box, dt=0.005, nsteps=50, n_pe=10, ckpt_every=10, **kw):
    """Convenience wrapper: eps and sigma may be python floats or 0-d tensors."""
    dev = x0.device
    eps_t = eps if torch.is_tensor(eps) else torch.tensor(float(eps), dtype=torch.float64, device=dev)
    sig_t = sigma if torch.is_tensor(sigma) else torch.tensor(float(sigma), dtype=torch.float64, device=dev)
    return LJTrajectory.apply(x0, v0, eps_t, sig_t, box, dt, nsteps, n_pe, ckpt_every,
                              kw.get("rc_over_sigma", 2.5), kw.get("margin", 0.5), kw.get("precision", ljmd.LJ_MIXED))
