"""Load stepping, checkpoints and the differentiable compliance around liblattice.so.

Orchestration only: predictor, Newton, adjoint and checkpoint I/O are library calls.
"""
from __future__ import annotations

import os

import torch

from .lattice import Lattice


def solve_load_path(lat: Lattice, case, opts=None, steps=None, checkpoint_dir=None, start=None, log=None):
    """Run load steps (start+1 .. steps) of ``case``; returns the final displacement.

    Step k prescribes the top face at -(k / n_steps) * strain * H.  The first step starts from
    the affine predictor, later steps from 2 u_{k-1} - u_{k-2} (library predictor).  With
    ``checkpoint_dir`` every converged step is saved (step, load, u_k, u_{k-1}); ``start`` =
    (step, u, u_prev) resumes after a saved step.
    """
    steps = case.n_steps if steps is None else steps
    k0, u1, u2 = (0, None, None) if start is None else start
    reports = []
    for k in range(k0 + 1, steps + 1):
        load = case.top_displacement(k)
        u = lat.lattice_predictor(load, u1, u2)
        rep = lat.newton_step(u, opts)
        if not rep.converged:
            raise RuntimeError(f"Newton did not converge at load step {k}: {rep.as_dict()}")
        reports.append(rep.as_dict())
        if log is not None:
            log(k, rep)
        if checkpoint_dir is not None:
            lat.lattice_checkpoint_save(os.path.join(checkpoint_dir, f"step_{k:04d}.ckpt"), k, load, u, u1)
        u2, u1 = u1, u
    return u1, reports


class Compliance(torch.autograd.Function):
    """J(theta): end compliance of the load path for per-cell shear-modulus factors theta.

    forward runs the load path on the GPU; backward calls adjoint_gradient (a transposed
    reduced-tangent solve with an exact-tangent defect correction) and returns dJ/dtheta.
    """

    @staticmethod
    def forward(ctx, theta, lat, case, opts):
        lat.lattice_set_mu_scale(theta.detach().cpu().double().numpy())
        u, _ = solve_load_path(lat, case, opts)
        g, J, rep = lat.adjoint_gradient(u, opts)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout * g.to(gout.device), None, None, None
