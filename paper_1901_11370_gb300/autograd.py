"""torch.autograd wrapper around the multigrid solve and its adjoint.

Forward: phi = A(eps)^-1 (f - b) by ``mg_solve`` (FP64).  Backward: given
dL/dphi, ``mg_adjoint`` solves A^T lambda = dL/dphi and returns
dL/df = lambda and dL/deps from the harmonic face coefficients.  Only phi at
the converged state is kept; the adjoint solve is recomputed, not taped.
"""
import torch


class MGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tree, f, eps, rel_tol=1e-12, max_cycles=60, adj_cycles=16):
        if eps is not None:
            tree.set_eps(eps.detach().contiguous())
        tree.set_rhs(f.detach().contiguous())
        tree.set_phi(torch.zeros_like(f))
        tree.solve(rel_tol, max_cycles, fmg_first=True, raise_on_fail=False)
        phi = tree.get_phi()
        ctx.tree = tree
        ctx.adj_cycles = adj_cycles
        ctx.has_eps = eps is not None
        ctx.save_for_backward(phi)
        return phi

    @staticmethod
    def backward(ctx, g):
        (phi,) = ctx.saved_tensors
        tree = ctx.tree
        tree.set_phi(phi)
        dLdf, dLde = tree.adjoint(g.contiguous(), n_cycles=ctx.adj_cycles, want_eps=ctx.has_eps)
        return None, dLdf, (dLde if ctx.has_eps else None), None, None, None


class CleanB(torch.autograd.Function):
    """Divergence cleaning B_new = B - grad A^+ P div B (Sec. 4.1) on a
    uniform periodic Cartesian mesh.  There the central gradient and
    divergence satisfy G^T = -D and the zero-mean solve and the mean
    projection P are symmetric, so the map is self-adjoint: the backward
    pass applies the same cleaning to the incoming gradient."""

    @staticmethod
    def forward(ctx, tree, B, rel_tol=1e-12, max_cycles=80):
        Bn, _, _, _ = tree.clean(B.detach(), rel_tol, max_cycles)
        ctx.tree, ctx.rel_tol, ctx.max_cycles = tree, rel_tol, max_cycles
        return Bn

    @staticmethod
    def backward(ctx, g):
        gB, _, _, _ = ctx.tree.clean(g.contiguous(), ctx.rel_tol, ctx.max_cycles)
        return None, gB, None, None
