"""torch.autograd.Function around the steady solve and its adjoint.

forward: build the HFDIB problem on the given lambda, converge it with
hfdib_solve_steady and return the objective J (pressure drop or drag) as a
0-d tensor.  backward: hfdib_adjoint_grad, the frozen-turbulence discrete
adjoint of that converged state, gives dJ/dlambda; it is multiplied by the
incoming gradient.  Both steps run in the library's CUDA kernels; this module
only passes pointers.

Typical use (topology optimisation over many designs):

    lam = torch.tensor(case["lam"], device="cuda", requires_grad=True)
    J = pressure_drop(lam, case)
    J.backward()          # lam.grad = dJ/dlambda

Many designs at once (grid sizes may differ): pressure_drops(lams, cases)
solves all of them together as one batch (hfdib_create_batch: one launch per
phase for all designs, the stop test on the device) and returns the vector
of their objectives; its backward pass runs the adjoint of every design.
"""
from __future__ import annotations

import torch

from .hfdib import BatchSolver, Solver


class SteadyRANS(torch.autograd.Function):
    """J(lambda) = pressure drop of the converged steady state."""

    @staticmethod
    def forward(ctx, lam, case, solve_tol, max_sweeps, adj_tol, adj_max_iter, opts, objective="pressure_drop"):
        c = dict(case)
        c["lam"] = lam.detach().to(torch.float64)
        s = Solver(c, device=lam.device, **opts)
        rc, it, res = s.solve(tol=solve_tol, max_iter=max_sweeps, check_every=20)
        if rc != 0:
            s.close()
            raise RuntimeError("steady solve did not reach %g in %d sweeps (status %d)" % (solve_tol, it, rc))
        ctx.solver = s
        ctx.adj = (adj_tol, adj_max_iter, objective)
        ctx.lam_shape = lam.shape
        return torch.tensor(s.objective(objective), dtype=torch.float64, device=lam.device)

    @staticmethod
    def backward(ctx, gout):
        s = ctx.solver
        tol, max_iter, objective = ctx.adj
        try:
            J, g, it, ch, rc = s.adjoint_grad(tol=tol, max_iter=max_iter, objective=objective)
        finally:
            s.close()
            ctx.solver = None
        if rc != 0:
            raise RuntimeError("adjoint did not converge to %g in %d iterations (change %.2e)" % (tol, it, ch))
        return gout * g.reshape(ctx.lam_shape), None, None, None, None, None, None, None


def pressure_drop(lam, case, solve_tol=1e-11, max_sweeps=40000, adj_tol=1e-10, adj_max_iter=20000, **opts):
    """Differentiable pressure drop of the case with indicator `lam` (a CUDA
    float64 tensor shaped (nz, ny, nx)); `opts` are hfdib options."""
    return SteadyRANS.apply(lam, case, solve_tol, max_sweeps, adj_tol, adj_max_iter, opts)


def drag(lam, case, solve_tol=1e-11, max_sweeps=40000, adj_tol=1e-10, adj_max_iter=20000, **opts):
    """Differentiable drag (x force of the fluid on the body) of the case with
    indicator `lam`; see pressure_drop."""
    return SteadyRANS.apply(lam, case, solve_tol, max_sweeps, adj_tol, adj_max_iter, opts, "drag")


class SteadyRANSBatch(torch.autograd.Function):
    """J_b(lambda_b), b = 0..B-1: the B steady states are converged together
    by one batch (hfdib_batch_solve_steady), and the backward pass gives each
    design's dJ_b/dlambda_b by hfdib_adjoint_grad on that design."""

    @staticmethod
    def forward(ctx, cases, solve_tol, max_sweeps, adj_tol, adj_max_iter, opts, objective, *lams):
        cs = [dict(c, lam=l.detach().to(torch.float64)) for c, l in zip(cases, lams)]
        bs = BatchSolver(cs, device=str(lams[0].device), **opts)
        rc, its, res = bs.solve(tol=solve_tol, max_iter=max_sweeps)
        if rc != 0:
            bs.close()
            worst = res[:, :6].max(axis=1)
            late = ", ".join("%d: %.1e after %d" % (i, worst[i], its[i]) for i in range(len(cs))
                             if not worst[i] <= solve_tol)
            raise RuntimeError("batch solve did not reach %g in %d sweeps (status %d); design: max scaled "
                               "residual after sweeps -- %s" % (solve_tol, max_sweeps, rc, late))
        ctx.batch = bs
        ctx.adj = (adj_tol, adj_max_iter, objective)
        ctx.shapes = [l.shape for l in lams]
        ctx.sweeps = [int(v) for v in its]
        J = [bs.problem(i).objective(objective) for i in range(len(cs))]
        return torch.tensor(J, dtype=torch.float64, device=lams[0].device)

    @staticmethod
    def backward(ctx, gout):
        bs = ctx.batch
        tol, max_iter, objective = ctx.adj
        grads = []
        try:
            for i in range(bs.B):
                J, g, it, ch, rc = bs.problem(i).adjoint_grad(tol=tol, max_iter=max_iter, objective=objective)
                if rc != 0:
                    raise RuntimeError("adjoint of design %d did not converge to %g in %d iterations (change %.2e)"
                                       % (i, tol, it, ch))
                grads.append(gout[i] * g.reshape(ctx.shapes[i]))
        finally:
            bs.close()
            ctx.batch = None
        return (None,) * 7 + tuple(grads)


def pressure_drops(lams, cases, solve_tol=1e-11, max_sweeps=40000, adj_tol=1e-10, adj_max_iter=20000,
                   objective="pressure_drop", **opts):
    """Differentiable objectives (pressure drop by default) of B designs with
    indicators `lams` (CUDA float64 tensors shaped like each case's grid),
    solved together as one batch; returns a tensor of B values."""
    return SteadyRANSBatch.apply(list(cases), solve_tol, max_sweeps, adj_tol, adj_max_iter, opts, objective,
                                 *lams)
