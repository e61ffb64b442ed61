"""Differentiable forms of the MMGKS-OF operators for torch.autograd.

Each forward and each backward pass is one call into the C ABI (hand-written
sm_103a kernels); this module only allocates outputs and routes gradients:

  project(p, u)               b = H u                      (Sec. 2.1)
      backward: du = H^T db                                 (mof_apply_AT)
  flow_residual(p, u, s, sr)  r = Mhat(s, s') u            (Sec. 2.3, Sec. 3)
      backward: du  = Mhat(s, s')^T dr                      (mof_apply_flowT)
                ds, dsr = velocity VJP of Mhat(s, s') u      (mof_apply_flow_ds)

The velocity derivative is that of the clipped bilinear warp: the bilinear
slope on the forward pass's cell, zero along an axis where the sample point is
clipped (derivative from the right at integer sample positions). Tensors are
CUDA tensors of the problem's precision, flat or of any shape with the
problem's element counts; gradients come back flat.
"""
import torch

from . import api


def _dtype(p):
    return torch.float64 if p.precision == api.MOF_FP64 else torch.float32


def _flat(x):
    return x.contiguous().reshape(-1)


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, p):
        ctx.p = p
        b = torch.empty(p.m, dtype=u.dtype, device=u.device)
        api.mof_apply_A(p, _flat(u), b)
        return b

    @staticmethod
    def backward(ctx, db):
        p = ctx.p
        du = torch.empty(p.n, dtype=db.dtype, device=db.device)
        api.mof_apply_AT(p, _flat(db), du)
        return du, None


class _FlowResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, s, sr, p):
        u, s, sr = _flat(u), _flat(s), _flat(sr)
        ctx.p = p
        ctx.save_for_backward(u, s, sr)
        r = torch.empty(2 * (p.nt - 1) * p.nx * p.ny, dtype=u.dtype, device=u.device)
        api.mof_apply_flow(p, u, s, sr, r)
        return r

    @staticmethod
    def backward(ctx, dr):
        p = ctx.p
        u, s, sr = ctx.saved_tensors
        dr = _flat(dr)
        du = gs = gsr = None
        if ctx.needs_input_grad[0]:
            du = torch.empty_like(u)
            api.mof_apply_flowT(p, dr, s, sr, du)
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            gs, gsr = torch.empty_like(s), torch.empty_like(sr)
            api.mof_apply_flow_ds(p, u, s, sr, dr, gs, gsr)
        return du, gs, gsr, None


def project(p, u):
    """H u for a problem p, differentiable in u."""
    if u.dtype != _dtype(p):
        raise TypeError("u must be %s for this problem" % _dtype(p))
    return _Project.apply(u, p)


def flow_residual(p, u, s, sr):
    """Mhat(s, s') u for a problem p, differentiable in u, s and sr."""
    for name, t in (("u", u), ("s", s), ("sr", sr)):
        if t.dtype != _dtype(p):
            raise TypeError("%s must be %s for this problem" % (name, _dtype(p)))
    return _FlowResidual.apply(u, s, sr, p)
