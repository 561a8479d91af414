"""torch.autograd.Function around the checkpointed adjoint-state gradient.

phi(m) = sum over shots of 1/2 ||d_sim(m) - d_obs||^2 with m = 1/c^2
(Sec. 6).  forward() runs forward modelling and the FP64 misfit in the
library (no adjoint, so line searches stay cheap); backward() runs the
library's checkpointed, optionally compressed adjoint (Sec. 3, Sec. 4) and
returns grad_output * dphi/dm, summed over shots in FP64 and rounded once.
"""
import torch

from . import ckfwi as C


class CheckpointedMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, model, shots, d_obs_list, opts):
        if not (m.is_cuda and m.dtype == torch.float32):
            raise ValueError("m must be a float32 CUDA tensor on the model's total grid")
        md = m.detach().contiguous()
        model.set_model(md, kind=C.SLOWNESS2)
        phi = 0.0
        for shot, d in zip(shots, d_obs_list):
            phi += model.misfit(shot, d)
        ctx.model, ctx.shots, ctx.d_obs, ctx.opts = model, shots, d_obs_list, dict(opts)
        ctx.save_for_backward(md)
        return torch.tensor(phi, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, grad_out):
        (m,) = ctx.saved_tensors
        scale = float(grad_out)
        if scale == 0.0:
            # the library reads a scale of 0 as 1; a zero upstream gradient
            # needs no adjoint run
            return torch.zeros_like(m), None, None, None, None
        ctx.model.set_model(m, kind=C.SLOWNESS2)
        g = torch.empty_like(m)
        opts = dict(ctx.opts)
        slots = opts.pop("ckpt_slots")
        ctx.model.batch_gradient(ctx.shots, ctx.d_obs, slots, grad_kind=C.SLOWNESS2,
                                 grad_scale=scale, grad_f32=True, grad_sum=g, **opts)
        return g, None, None, None, None


def misfit(m, model, shots, d_obs_list, ckpt_slots, **opts):
    """Differentiable total misfit of `shots` at slowness-squared m."""
    return CheckpointedMisfit.apply(m, model, shots, d_obs_list, dict(opts, ckpt_slots=ckpt_slots))


def steepest_descent(m0, model, shots, d_obs_list, iterations, ckpt_slots, step=0.05, m_min=None, m_max=None,
                     backtrack=6, stop_on_stall=False, **opts):
    """Steepest descent m <- clip(m - alpha g / max|g|), starting from
    alpha = step * max|m| and halving alpha until the misfit decreases
    (the paper names steepest descent, Sec. 6; the step rule is this
    driver's).  Each trial costs one forward-only misfit.  With
    stop_on_stall, the iterations end when no trial lowers the misfit (the
    next iteration would repeat the same search).  Returns (m, misfit
    history)."""
    m = m0.detach().clone()
    hist = []
    phi_m = None
    for _ in range(iterations):
        x = m.clone().requires_grad_(True)
        phi = misfit(x, model, shots, d_obs_list, ckpt_slots, **opts)
        (g,) = torch.autograd.grad(phi, x)
        phi_m = float(phi.detach())
        hist.append(phi_m)
        with torch.no_grad():
            d = g / g.abs().max()
            alpha = step * float(m.abs().max())
            for _ in range(backtrack):
                trial = m - alpha * d
                if m_min is not None or m_max is not None:
                    trial.clamp_(min=m_min, max=m_max)
                phi_t = float(misfit(trial, model, shots, d_obs_list, ckpt_slots, **opts))
                if phi_t < phi_m:
                    m = trial
                    phi_m = phi_t
                    break
                alpha *= 0.5
            else:
                if stop_on_stall:
                    break
    hist.append(phi_m if phi_m is not None else float(misfit(m, model, shots, d_obs_list, ckpt_slots, **opts)))
    return m, hist
