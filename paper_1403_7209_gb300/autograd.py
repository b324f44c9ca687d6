"""R(q, n) as a differentiable torch function backed by the adjoint kernels.

``residual(solver, q, n)`` returns the edge-loop residual R (6, N) of the
state q (6, N) and the edge normals n (3, E) (library numbering, FP64 CUDA
tensors).  Its backward pass runs the hand-written adjoint edge loops: for
an incoming gradient lam = dL/dR it returns qbar = lam . dR/dq and
nbar = lam . dR/dn.  Forward-mode AD (``torch.autograd.forward_ad``) runs
the tangent-linear edge loops: dR = dR/dq . qd + dR/dn . nd.  The forward
pass keeps the node gradients G (node data, 18 values per node); the edge
states are recomputed from q, G and n instead of being stored.
"""
from __future__ import annotations

import torch


class ResidualFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, n, solver, order):
        s = solver
        s.rebind("q", q.detach().contiguous())
        s.rebind("n", n.detach().contiguous())
        out = torch.empty_like(s.t["R"])
        s.rebind("R", out)
        G = torch.empty_like(s.t["G"])
        s.rebind("G", G)
        s.residual(order)
        ctx.solver, ctx.order = s, order
        ctx.save_for_backward(q, n, G)
        ctx.save_for_forward(q, n, G)
        return out

    @staticmethod
    def jvp(ctx, q_t, n_t, solver_t, order_t):
        s = ctx.solver
        q, n, G = ctx.saved_tensors
        s.rebind("q", q.detach().contiguous())
        s.rebind("n", n.detach().contiguous())
        s.rebind("G", G)
        s.rebind("qd", (q_t if q_t is not None else torch.zeros_like(q)).detach().double().contiguous())
        s.rebind("nd", (n_t if n_t is not None else torch.zeros_like(n)).detach().double().contiguous())
        Rd = torch.empty_like(s.t["Rd"])
        s.rebind("Rd", Rd)
        s.tangent(ctx.order, recompute_gradient=False)
        return Rd

    @staticmethod
    def backward(ctx, grad_r):
        s = ctx.solver
        q, n, G = ctx.saved_tensors
        s.rebind("q", q.detach().contiguous())
        s.rebind("n", n.detach().contiguous())
        s.rebind("G", G)
        s.rebind("lam", grad_r.detach().double().contiguous())
        qbar = torch.empty_like(s.t["qbar"])
        nbar = torch.empty_like(s.t["nbar"])
        s.rebind("qbar", qbar)
        s.rebind("nbar", nbar)
        s.adjoint(ctx.order, recompute_gradient=False)
        return qbar, nbar, None, None


def residual(solver, q, n, order=2):
    """Differentiable R(q, n); the solver must be built with adjoint=True."""
    if not solver.has_adjoint:
        raise ValueError("build the EdgeSolver with adjoint=True")
    if solver.visc is not None or solver.limiter != "van_albada":
        raise ValueError("the adjoint and tangent loops cover the inviscid residual with the "
                         "van Albada limiter only")
    return ResidualFn.apply(q, n, solver, order)
