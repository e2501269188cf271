"""PyTorch autograd wrappers over the C-ABI (marshalling only; every derivative is one
of libchns's kernels or solvers).

* ``Residual``      R(U^k, U^{k+1}; Cn): backward = J^T w kernel (with the U^k and Cn
                    parts), forward mode = J x kernel (tangent of U^{k+1} only).
* ``ImplicitStep``  U^{k+1}(U^k, Cn) defined by R = 0 (Section 3.4): forward = Newton,
                    backward = the adjoint solve J^T lambda = g (implicit function theorem).
* ``InitialMu``     mu^0(phi^0, Cn) from M mu^0 = b(phi^0; Cn): backward = mass solve and
                    the reverse mode of b.
* ``FreeEnergy``    the free-energy part of E_tot at one time level.
* ``rollout``       a multi-step rollout with checkpointed recomputation.
"""
import ctypes

import torch
import torch.utils.checkpoint

from . import (ChnsError, Params, free_energy_grad, initial_mu, jvp, mass_solve, mu_rhs_vjp, newton_step,
               residual, step_adjoint, vjp)


def with_cn(prm, Cn):
    """Copy of a Params struct with Cn replaced (Cn may be a 0-d tensor)."""
    q = Params()
    ctypes.pointer(q)[0] = prm
    q.Cn = float(Cn)
    return q


class Residual(torch.autograd.Function):
    """R(U^k, U^{k+1}; Cn) with reverse mode (J^T w kernel) and forward mode (J x kernel,
    tangents of U^{k+1} only); usable under torch.func transforms."""

    @staticmethod
    def forward(mesh, prm, U_old, U_new, Cn):
        return residual(mesh, with_cn(prm, Cn), U_old.contiguous(), U_new.contiguous())

    @staticmethod
    def setup_context(ctx, inputs, output):
        mesh, prm, U_old, U_new, Cn = inputs
        ctx.mesh, ctx.prm = mesh, with_cn(prm, Cn)
        ctx.save_for_backward(U_old, U_new)
        ctx.save_for_forward(U_old, U_new)

    @staticmethod
    def backward(ctx, gR):
        U_old, U_new = ctx.saved_tensors
        gn, go, gc = vjp(ctx.mesh, ctx.prm, U_old.contiguous(), U_new.contiguous(), gR.contiguous())
        return None, None, go, gn, gc.reshape(())

    @staticmethod
    def jvp(ctx, _m, _p, t_old, t_new, t_cn):
        U_old, U_new = ctx.saved_tensors
        for t in (t_old, t_cn):
            if t is not None and bool(torch.any(t != 0)):
                raise NotImplementedError("forward mode supports tangents of U^{k+1} only")
        if t_new is None:
            return torch.zeros_like(U_new)
        return jvp(ctx.mesh, ctx.prm, U_old.contiguous(), U_new.contiguous(), t_new.contiguous())


class ImplicitStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, prm, opts, adj_opts, U_old, Cn):
        p = with_cn(prm, Cn)
        U_new, st = newton_step(mesh, p, opts, U_old.contiguous())
        ctx.mesh, ctx.prm, ctx.adj_opts = mesh, p, adj_opts
        ctx.save_for_backward(U_old, U_new)
        return U_new

    @staticmethod
    def backward(ctx, g):
        U_old, U_new = ctx.saved_tensors
        _, go, gc, _ = step_adjoint(ctx.mesh, ctx.prm, ctx.adj_opts, U_old.contiguous(), U_new.contiguous(),
                                    g.contiguous())
        return None, None, None, None, go, gc.reshape(())


class InitialMu(torch.autograd.Function):
    """U with its mu field replaced by the discrete mu^0 of its phi (the incoming mu is
    ignored, so it receives no gradient)."""

    @staticmethod
    def forward(ctx, mesh, prm, U, Cn):
        p = with_cn(prm, Cn)
        out = U.detach().clone().contiguous()
        initial_mu(mesh, p, out)
        ctx.mesh, ctx.prm = mesh, p
        ctx.save_for_backward(out)
        return out

    @staticmethod
    def backward(ctx, g):
        (U,) = ctx.saved_tensors
        d = ctx.mesh.dim
        lam = mass_solve(ctx.mesh, g[:, d + 2].contiguous())
        g_phi, dcn = mu_rhs_vjp(ctx.mesh, ctx.prm, U, lam)
        gU = g.clone()
        gU[:, d + 2] = 0.0
        gU[:, d + 1] += g_phi
        return None, None, gU, torch.tensor(dcn, dtype=torch.float64, device=g.device)


class FreeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, prm, U, Cn):
        from . import energy
        p = with_cn(prm, Cn)
        ctx.mesh, ctx.prm = mesh, p
        ctx.save_for_backward(U)
        return torch.tensor(energy(mesh, p, U.contiguous())[1], dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gE):
        (U,) = ctx.saved_tensors
        g, dcn = free_energy_grad(ctx.mesh, ctx.prm, U.contiguous())
        return None, None, gE * g, gE * torch.tensor(dcn, dtype=torch.float64, device=U.device)


def rollout(mesh, prm, opts, adj_opts, U0, Cn, n_steps, checkpoint_every=5):
    """Free energy after ``n_steps`` implicit steps from the state U0 (its mu field is
    recomputed from phi and Cn).  Every ``checkpoint_every`` steps form one segment whose
    states are recomputed during the backward pass instead of stored."""
    U = InitialMu.apply(mesh, prm, U0, Cn)
    failed = []

    def segment(U_in, Cn_in, k):
        # a solver failure is re-raised after checkpoint() returns: an exception thrown
        # through the non-reentrant checkpoint leaves its saved-tensor hooks installed
        for _ in range(k):
            try:
                U_in = ImplicitStep.apply(mesh, prm, opts, adj_opts, U_in, Cn_in)
            except ChnsError as e:
                failed.append(e)
                break
        return U_in

    done = 0
    while done < n_steps:
        k = min(checkpoint_every, n_steps - done)
        if torch.is_grad_enabled() and checkpoint_every > 0:
            U = torch.utils.checkpoint.checkpoint(segment, U, Cn, k, use_reentrant=False)
        else:
            U = segment(U, Cn, k)
        if failed:
            raise failed[0]
        done += k
    return FreeEnergy.apply(mesh, prm, U, Cn)
