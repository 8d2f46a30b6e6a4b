"""Deposited mass as a differentiable function of the initial concentration and the
settling velocity (torch.autograd), backed by the hand-written adjoint of the coupled
2D step in liblbm_wenoc.so.

``deposited_mass(c0, vs, nsteps, shape=..., lf_alpha=..., ...)`` returns the mass that
has crossed the floor after ``nsteps`` steps (Sec. 4, m_b) as a 0-d FP64 tensor.  When a
gradient is needed the forward pass already runs the checkpointed forward + reverse
sweep of the library (one call), keeps dJ/dc0 and dJ/dVs, and the backward pass only
scales them by the incoming gradient.  The Lax-Friedrichs alpha must be given
(``lf_alpha``) and stays fixed under a change of Vs.
"""
import torch

from . import lbm_wenoc as lw


class _DepositedMass(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c0, vs, cfg):
        shape, nsteps, segment, kw = cfg
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        sim = lw.Simulation(shape, settling_velocity=float(vs), **kw)
        try:
            if need:
                J, g, dvs = sim.deposit_gradient(c0.detach(), nsteps, segment)
                ctx.save_for_backward(g.to(c0.dtype).reshape(c0.shape),
                                      torch.tensor(dvs, dtype=torch.float64, device=c0.device))
            else:
                sim.init(c0.detach())
                sim.step(nsteps)
                J = sim.deposit
        finally:
            sim.close()
        return torch.tensor(J, dtype=torch.float64, device=c0.device)

    @staticmethod
    def backward(ctx, gout):
        g, dvs = ctx.saved_tensors
        gc = (gout.to(g.dtype) * g) if ctx.needs_input_grad[0] else None
        gv = (gout * dvs).to(torch.float64) if ctx.needs_input_grad[1] else None
        return gc, gv, None


def deposited_mass(c0, vs, nsteps, shape, segment=None, **params):
    """Differentiable deposited mass.  c0: CUDA tensor of the grid's shape (ny, nx);
    vs: float or 0-d tensor (settling velocity); shape = (nx, ny); params: the other
    keyword arguments of ``make_params`` (lf_alpha > 0 required for gradients)."""
    if not isinstance(vs, torch.Tensor):
        vs = torch.tensor(float(vs), dtype=torch.float64)
    return _DepositedMass.apply(c0, vs, (tuple(shape), int(nsteps), segment, params))
