"""torch.autograd wrapper of the pseudofermion action

    S(U, phi) = sum_v Re phi_v^dag (D^dag D)^-1 phi_v,   D = D_W, D_S or D_B

(the paper has no differentiation; this grows its Wilson, staggered and
Brillouin operators and CG solver into a differentiable layer; for D_B the
link gradient runs back through the path-averaged W links of Tab. off-axis).  Forward: one CG solve of
D^dag D psi = phi (``dirac_solve`` with DIRAC_CG_HPD) and S = Re <phi, psi>
from the library's dot product.  Backward: the adjoint solve, recomputed
instead of stored (D^dag D is Hermitian, so the adjoint system is the forward
one; no Krylov vectors are kept between the passes), then chi = D psi and the
link gradient from ``dirac_force``:

    dS/dU   = G   with dS = Re sum conj(G) dU     (torch's convention for complex inputs)
    dS/dphi = 2 psi

All arithmetic runs in libdirac kernels; this module only marshals tensors.
"""
import torch

from . import dirac as D


class _Action(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, holder, m0, tol, maxit, prec, bc, save_solution):
        op = holder.op_for(U, phi, prec, bc)
        x, st = op.solve(op.to_prec(phi), m0=m0, solver=D.CG_HPD, tol=tol, maxit=maxit)
        if st["status"] != 0:
            raise RuntimeError("pseudofermion solve did not converge: %s" % st)
        S = op.dot(op.to_prec(phi), x).real.sum()
        ctx.holder, ctx.m0, ctx.tol, ctx.maxit, ctx.prec, ctx.bc = holder, m0, tol, maxit, prec, bc
        ctx.solution = x if save_solution else None
        ctx.save_for_backward(U, phi)
        holder.last_stats = st
        return S.to(torch.float64)

    @staticmethod
    def backward(ctx, gS):
        U, phi = ctx.saved_tensors
        op = ctx.holder.op_for(U, phi, ctx.prec, ctx.bc)
        x = ctx.solution
        if x is None:   # adjoint solve, recomputed
            x, st = op.solve(op.to_prec(phi), m0=ctx.m0, solver=D.CG_HPD, tol=ctx.tol, maxit=ctx.maxit)
            if st["status"] != 0:
                raise RuntimeError("adjoint solve did not converge: %s" % st)
        chi = op.apply(x, m0=ctx.m0)
        G = op.force(x, chi, mode=D.FORCE_GRAD)
        gU = (gS.to(G.real.dtype) * G).to(U.dtype) if ctx.needs_input_grad[0] else None
        gphi = (2 * gS) * op.to_complex(x).to(phi.dtype) if ctx.needs_input_grad[1] else None
        return gU, gphi, None, None, None, None, None, None, None


class _Stout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, rho, nsteps):
        ctx.rho, ctx.nsteps = rho, nsteps
        ctx.save_for_backward(U)
        return D.stout_smear(U.detach().contiguous(), rho, nsteps)

    @staticmethod
    def backward(ctx, gV):
        U, = ctx.saved_tensors
        gU = D.stout_backward(U.detach().contiguous(), gV.contiguous().to(U.dtype), ctx.rho, ctx.nsteps)
        return gU, None, None


def stout_smear(U, rho=0.12, nsteps=3):
    """Differentiable stout smearing V(U) (dirac_stout_smear forward,
    dirac_stout_backward for the gradient): composes with PseudofermionAction
    to give the force of an operator built from smeared links."""
    return _Stout.apply(U, float(rho), int(nsteps))


class PseudofermionAction:
    """Differentiable S(U, phi) for the Wilson (default), staggered or
    Brillouin operator on one lattice shape.

    The operator handle is created on first use and its links refreshed from
    U on every call (``dirac_op_update_links``)."""

    def __init__(self, m0, bc=(1, 1, 1, 1), prec=D.F32, tol=1e-8, maxit=20000, save_solution=False, kind=D.WILSON):
        if kind not in (D.WILSON, D.STAGGERED, D.BRILLOUIN):
            raise ValueError("the force is derived for D_W, D_S and D_B")
        self.kind = kind
        self.m0, self.bc, self.prec = float(m0), tuple(bc), prec
        self.tol, self.maxit, self.save_solution = tol, maxit, save_solution
        self.op = None
        self.last_stats = None

    def op_for(self, U, phi, prec, bc):
        nv = phi.shape[-1]
        if self.op is None or self.op.nv != nv or self.op.dims != (U.shape[3], U.shape[2], U.shape[1], U.shape[0]):
            self.op = D.DiracOp(self.kind, U.detach(), nv, bc, prec)
        else:
            self.op.update_links(U.detach())
        return self.op

    def __call__(self, U, phi):
        return _Action.apply(U, phi, self, self.m0, self.tol, self.maxit, self.prec, self.bc, self.save_solution)

    def force(self, U, phi):
        """Traceless anti-hermitian force F_mu(n) (dS/deps = Re sum tr[X F] for U -> exp(eps X) U)."""
        op = self.op_for(U, phi, self.prec, self.bc)
        x, st = op.solve(op.to_prec(phi), m0=self.m0, solver=D.CG_HPD, tol=self.tol, maxit=self.maxit)
        chi = op.apply(x, m0=self.m0)
        return op.force(x, chi, mode=D.FORCE_TA)
