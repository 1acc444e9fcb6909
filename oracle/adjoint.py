"""Adjoint gradient of end compliance w.r.t. per-cell shear-modulus factors (oracle, FP64).

Not in the paper; derived here from the discrete equilibrium.  With mu_s = theta_s mu, the
final state u = (u_F, u_D) solves r_F(u, theta) = 0 (Eq. residualvector on the free DOFs) and the
objective is the reaction work J = u_D . f_D(u, theta) over the Dirichlet DOFs.  Then

    K_FF lambda = K_FD u_D,     dJ/dtheta_s = w^T A^s f_mu^s(u^s),   w = [-lambda ; u_D],

where f_mu^s = d f^{int,s} / d theta_s is the internal force of Eq. (internalloadvec) evaluated
with the stress mu/J (b - I) alone (Eq. sig_eq is linear in mu).  The linear solve is direct.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import cell as C


def gradient(prob, u, mu=None):
    mu = prob.mu_cells if mu is None else mu
    free, fixed = prob.free, prob.fixed
    K = prob.tangent(u, mu)
    uD = u[fixed]
    rhs = K[free][:, fixed] @ uD
    lam = spla.splu(K[free][:, free].tocsc()).solve(rhs)
    w = np.zeros(prob.n_dof)
    w[free] = -lam
    w[fixed] = uD
    base = prob.case.mu
    f_mu = C.internal_force(prob.cell, prob.local(u), np.full(prob.lat.n_cells, base), 0.0)
    ws = w[prob.cell_dofs]
    return np.einsum("sk,sk->s", ws, f_mu.reshape(prob.lat.n_cells, -1))
