"""torch.autograd wrappers around the multigrid solve and its adjoint.

MGSolve -- forward: phi = A(eps)^-1 (f - b) by ``mg_solve`` (FP64); on a
problem without Dirichlet faces f must be compatible and phi is the
zero-mean solution.  Backward: given dL/dphi, ``mg_adjoint_solve`` solves
A^T lambda = dL/dphi and returns dL/df = lambda and dL/deps through the
harmonic face coefficients.  Only phi at the converged state is kept; the
adjoint solve is recomputed, not taped.  Both solves raise MGError when they
do not reach their tolerance, so a gradient is never returned from an
unconverged state.

CleanB -- divergence cleaning B_new = B - grad phi, Lap phi = div B
(Sec. 4.1); backward is ``mg_clean_adjoint`` (the transposed divergence,
gradient and operator on any Cartesian mesh, refinement faces included).
"""
import torch


class MGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tree, f, eps, rel_tol=1e-12, max_cycles=80, adj_tol=1e-12):
        if eps is not None:
            tree.set_eps(eps.detach().contiguous())
        tree.set_rhs(f.detach().contiguous())
        tree.set_phi(torch.zeros_like(f))
        tree.solve(rel_tol, max_cycles, fmg_first=True)  # raises MGError when not converged
        phi = tree.get_phi()
        ctx.tree = tree
        ctx.adj_tol = adj_tol
        ctx.max_cycles = max_cycles
        ctx.has_eps = eps is not None
        ctx.save_for_backward(phi)
        return phi

    @staticmethod
    def backward(ctx, g):
        (phi,) = ctx.saved_tensors
        tree = ctx.tree
        tree.set_phi(phi)
        dLdf, dLde = tree.adjoint(g.contiguous(), want_eps=ctx.has_eps, rel_tol=ctx.adj_tol,
                                  max_cycles=ctx.max_cycles)
        return None, dLdf, (dLde if ctx.has_eps else None), None, None, None


class CleanB(torch.autograd.Function):
    """Divergence cleaning B_new = B - grad A^+ P div B (Sec. 4.1); the
    backward pass is the exact vector-Jacobian product of the discrete map."""

    @staticmethod
    def forward(ctx, tree, B, rel_tol=1e-12, max_cycles=80):
        Bn, _, _, rel = tree.clean(B.detach(), rel_tol, max_cycles)
        if not rel <= rel_tol:
            from ._lib import MGError
            raise MGError(-4, "cleaning solve did not reach %g (relative residual %g)" % (rel_tol, rel))
        ctx.tree, ctx.rel_tol, ctx.max_cycles = tree, rel_tol, max_cycles
        return Bn

    @staticmethod
    def backward(ctx, g):
        gB = ctx.tree.clean_adjoint(g.contiguous(), ctx.rel_tol, ctx.max_cycles)
        return None, gB, None, None
