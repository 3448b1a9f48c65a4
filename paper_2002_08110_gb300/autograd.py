"""Differentiation through LSRK(5,4) time integration of the DG operator.

``RKForward.apply(u0, dg, dt, nsteps, prec, checkpoint_every)`` returns
u(T) = Phi^nsteps(u0), Phi = one LSRK(5,4) step of du/dt = L u with
L = M^{-1} A (the library's fused stages).  Its backward applies the adjoint
step Phi^T = R(dt L)^T = R(dt L^T) (the step map is the stability polynomial
R of dt L, and R(X)^T = R(X^T)) nsteps times with the library's transposed
operator L^T = M L(-a) M^{-1}.

Checkpointing: the forward keeps the state every ``checkpoint_every`` steps.
The backward walks the segments in reverse; for each one it recomputes the
segment forward from its checkpoint (where an adjoint of a state-dependent
operator would take its states) and checks that the recomputed end state
equals the next stored checkpoint bit for bit (the kernels are
deterministic), then runs the segment's adjoint steps.  For the linear,
autonomous operator of this library the adjoint steps do not read the
recomputed states; the recomputation is the memory/compute trade the pattern
exists for, and its consistency check guards the stored trajectory.

``misfit_gradient`` is the gradient of 0.5 * ||u(T) - u_target||^2 with
respect to u0.

``VPForward`` / ``vp_misfit_gradient``: the same for the FP64 Vlasov-Poisson
steps (dim_x = 1), whose stage operator depends on the state through the
field.  There the adjoint of each step needs that step's states: the
backward recomputes each segment from its checkpoint one step at a time,
keeps the segment's step-start states, and runs the adjoint steps
(``dg_vp_step_adjoint``: the step's stages recomputed and transposed) in
reverse from them.
"""
import torch

from ._lib import PREC_FP32, PREC_FP64  # noqa: F401


class CheckpointMismatch(RuntimeError):
    """A recomputed segment did not end on the stored checkpoint bit for bit."""


class RKForward(torch.autograd.Function):
    """u(T) = Phi^nsteps(u0) with a checkpointed adjoint backward (module doc)."""

    @staticmethod
    def forward(ctx, u0, dg, dt, nsteps, prec, checkpoint_every):
        """nsteps LSRK(5,4) steps of the handle ``dg``; keeps every
        ``checkpoint_every``-th state for the backward."""
        if checkpoint_every < 1:
            raise ValueError("checkpoint_every must be >= 1")
        u = u0.detach().to(torch.float64).contiguous().clone()
        wdt = torch.float32 if prec == PREC_FP32 else torch.float64
        w0 = torch.empty(dg.n_dofs, dtype=wdt, device=u.device)
        w1 = torch.empty_like(w0)
        checkpoints = [u.clone()]
        done = 0
        while done < nsteps:
            seg = min(checkpoint_every, nsteps - done)
            dg.rk_step(u, dt, nsteps=seg, prec=prec, w0=w0, w1=w1)
            done += seg
            if done < nsteps:
                checkpoints.append(u.clone())
        ctx.dg, ctx.dt, ctx.nsteps, ctx.prec, ctx.every = dg, dt, nsteps, prec, checkpoint_every
        ctx.checkpoints = checkpoints
        ctx.final = u.clone()
        ctx.recomputed_segments = 0
        return u

    @staticmethod
    def backward(ctx, grad_out):
        """Phi^T applied nsteps times to grad_out, segment by segment in
        reverse, each segment recomputed from its checkpoint and checked."""
        dg, dt, prec, every = ctx.dg, ctx.dt, ctx.prec, ctx.every
        lam = grad_out.detach().to(torch.float64).contiguous().clone()
        wdt = torch.float32 if prec == PREC_FP32 else torch.float64
        w0 = torch.empty(dg.n_dofs, dtype=wdt, device=lam.device)
        w1 = torch.empty_like(w0)
        bounds = []
        s = 0
        while s < ctx.nsteps:
            bounds.append((s, min(s + every, ctx.nsteps)))
            s += every
        x = torch.empty_like(lam)
        for k in reversed(range(len(bounds))):
            a, b = bounds[k]
            # recompute the segment from its checkpoint (one graph-replayed
            # call); its end state must reproduce the next checkpoint exactly
            x.copy_(ctx.checkpoints[k])
            dg.rk_step(x, dt, nsteps=b - a, prec=prec, w0=w0, w1=w1)
            nxt = ctx.checkpoints[k + 1] if k + 1 < len(ctx.checkpoints) else ctx.final
            if not torch.equal(x, nxt):
                raise CheckpointMismatch(f"recomputed state of segment {k} differs from its checkpoint")
            ctx.recomputed_segments += 1
            # the segment's adjoint steps (identical steps R(dt L^T) for this
            # autonomous operator, so one call runs all of them)
            dg.rk_step(lam, dt, nsteps=b - a, prec=prec, adjoint=True, w0=w0, w1=w1)
        dg.check()
        return lam.to(grad_out.dtype), None, None, None, None, None


def final_state(u0, dg, dt, nsteps, prec=PREC_FP32, checkpoint_every=20):
    """u(T) as a differentiable function of u0."""
    return RKForward.apply(u0, dg, dt, nsteps, prec, checkpoint_every)


def misfit_gradient(u0, u_target, dg, dt, nsteps, prec=PREC_FP32, checkpoint_every=20):
    """(J, dJ/du0) for J = 0.5 ||u(T) - u_target||^2 (Euclidean DoF norm)."""
    x = u0.detach().clone().requires_grad_(True)
    uT = final_state(x, dg, dt, nsteps, prec, checkpoint_every)
    J = 0.5 * torch.sum((uT - u_target) ** 2)
    J.backward()
    return float(J.detach()), x.grad


class VPForward(torch.autograd.Function):
    """u(T) after nsteps FP64 Vlasov-Poisson steps, with a checkpointed
    adjoint backward (module doc)."""

    @staticmethod
    def forward(ctx, u0, dg, dt, nsteps, checkpoint_every):
        if checkpoint_every < 1:
            raise ValueError("checkpoint_every must be >= 1")
        u = u0.detach().to(torch.float64).contiguous().clone()
        w0 = torch.empty(dg.n_dofs, dtype=torch.float64, device=u.device)
        w1 = torch.empty_like(w0)
        checkpoints = [u.clone()]
        done = 0
        while done < nsteps:
            seg = min(checkpoint_every, nsteps - done)
            dg.vp_rk_step(u, dt, nsteps=seg, prec=PREC_FP64, w0=w0, w1=w1)
            done += seg
            if done < nsteps:
                checkpoints.append(u.clone())
        ctx.dg, ctx.dt, ctx.nsteps, ctx.every = dg, dt, nsteps, checkpoint_every
        ctx.checkpoints = checkpoints
        ctx.final = u.clone()
        return u

    @staticmethod
    def backward(ctx, grad_out):
        dg, dt, every = ctx.dg, ctx.dt, ctx.every
        lam = grad_out.detach().to(torch.float64).contiguous().clone()
        w0 = torch.empty(dg.n_dofs, dtype=torch.float64, device=lam.device)
        w1 = torch.empty_like(w0)
        bounds = []
        s = 0
        while s < ctx.nsteps:
            bounds.append((s, min(s + every, ctx.nsteps)))
            s += every
        for k in reversed(range(len(bounds))):
            a, b = bounds[k]
            # the segment's step-start states, recomputed from its checkpoint
            states = [ctx.checkpoints[k].clone()]
            for _ in range(b - a - 1):
                x = states[-1].clone()
                dg.vp_rk_step(x, dt, nsteps=1, prec=PREC_FP64, w0=w0, w1=w1)
                states.append(x)
            end = states[-1].clone()
            dg.vp_rk_step(end, dt, nsteps=1, prec=PREC_FP64, w0=w0, w1=w1)
            nxt = ctx.checkpoints[k + 1] if k + 1 < len(ctx.checkpoints) else ctx.final
            if not torch.equal(end, nxt):
                raise CheckpointMismatch(f"recomputed state of segment {k} differs from its checkpoint")
            for x in reversed(states):
                dg.vp_step_adjoint(x, lam, dt)
        dg.check()
        return lam.to(grad_out.dtype), None, None, None, None


def vp_final_state(u0, dg, dt, nsteps, checkpoint_every=10):
    """u(T) of the Vlasov-Poisson steps as a differentiable function of u0."""
    return VPForward.apply(u0, dg, dt, nsteps, checkpoint_every)


def vp_misfit_gradient(u0, u_target, dg, dt, nsteps, checkpoint_every=10):
    """(J, dJ/du0) for J = 0.5 ||u(T) - u_target||^2 through Vlasov-Poisson steps."""
    x = u0.detach().clone().requires_grad_(True)
    uT = vp_final_state(x, dg, dt, nsteps, checkpoint_every)
    J = 0.5 * torch.sum((uT - u_target) ** 2)
    J.backward()
    return float(J.detach()), x.grad
