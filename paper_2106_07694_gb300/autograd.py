"""Deposited mass as a differentiable function of the initial concentration and the
settling velocity (torch.autograd), backed by the hand-written adjoint of the coupled
2D step in liblbm_wenoc.so.

``deposited_mass(c0, vs, nsteps, shape=..., lf_alpha=..., ...)`` returns the mass that
has crossed the floor after ``nsteps`` steps (Sec. 4, m_b) as a 0-d FP64 tensor.  When a
gradient is needed the forward pass already runs the checkpointed forward + reverse
sweep of the library (one call), keeps dJ/dc0 and dJ/dVs, and the backward pass only
scales them by the incoming gradient.  The Lax-Friedrichs alpha must be given
(``lf_alpha``) and stays fixed under a change of Vs.

The handle and its adjoint workspace of the last configuration are kept for the next
call with the same configuration (an optimisation loop calls with the same sizes);
``release()`` frees them.
"""
import torch

from . import lbm_wenoc as lw


_cache = {}


def release():
    """Free the cached handle and workspace."""
    for sim, _ in _cache.values():
        sim.close()
    _cache.clear()


def _simulation(shape, vs, nsteps, segment, kw):
    key = (tuple(shape), float(vs), int(nsteps), segment, tuple(sorted(kw.items())))
    hit = _cache.get(key)
    if hit is None:
        release()
        sim = lw.Simulation(shape, settling_velocity=float(vs), **kw)
        seg = lw.default_segment(nsteps) if segment is None else int(segment)
        nbytes = lw.lbm_wenoc_gradient_workspace_bytes(sim.params, nsteps, seg)
        adj = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        grad = torch.empty(sim.grid, dtype=sim.dtype, device="cuda")
        hit = _cache[key] = (sim, (seg, adj, nbytes, grad))
    return hit


class _DepositedMass(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c0, vs, cfg):
        shape, nsteps, segment, kw = cfg
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        sim, (seg, adj, nbytes, grad) = _simulation(shape, vs, nsteps, segment, kw)
        c = c0.detach().to(sim.dtype).contiguous()
        if need:
            J, dvs = lw.lbm_wenoc_deposit_gradient(sim.handle, c, nsteps, seg, adj, nbytes, grad)
            ctx.save_for_backward(grad.to(c0.dtype).reshape(c0.shape).clone(),
                                  torch.tensor(dvs, dtype=torch.float64, device=c0.device))
        else:
            lw.lbm_wenoc_init(sim.handle, c)
            lw.lbm_wenoc_step(sim.handle, nsteps)
            J = lw.lbm_wenoc_deposited_mass(sim.handle)
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
