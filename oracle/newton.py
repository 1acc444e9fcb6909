"""Newton-Raphson with Armijo backtracking and load stepping (oracle, FP64).

Section 2.2.5: solve K(u^i) du = -r(u^i) (Eq. linsys) on the free DOFs, then take the smallest
m >= 0 with ||r(u + beta^m du)||_2 <= (1 - c beta^m) ||r(u)||_2, beta = 1/2, c = 1e-4; stop when
||r(u^{i+1})||_2 / ||r(u^0)||_2 <= tol.  The linear solve is a sparse direct LU (the paper's
"standard method", Section 4.2).

Readings where the paper is silent:
* a trial point with any quadrature point at det F <= 0 fails the Armijo test; m <= 30;
* load step k prescribes the top face at -(k / n_steps) * strain * H along the load axis;
* predictor: step 1 starts from the affine field u_axis = (delta_1 / H) X_axis, later steps
  from the linear extrapolation 2 u_{k-1} - u_{k-2}; Dirichlet values are then overwritten;
* r0 is the predictor's residual; an absolute floor of 1e-12 ||f_int(u)||_2 (all DOFs,
  reactions included) stops the iteration once the free residual is at round-off level
  (below it Armijo cannot find a decrease: the residual only changes by rounding).
"""
import dataclasses

import numpy as np
import scipy.sparse.linalg as spla

BETA = 0.5
C_ARMIJO = 1e-4
MAX_M = 30


@dataclasses.dataclass
class NewtonReport:
    iterations: int
    residual_history: list
    line_search: list
    converged: bool


def predictor(prob, step, u_prev, u_prev2):
    """Initial guess of load step ``step``: affine field for step 1, else 2 u_{k-1} - u_{k-2}.

    u_0 (before step 1) is the undeformed state 0, so step 2 starts from 2 u_1.
    """
    lat = prob.lat
    if step == 1 or u_prev is None:
        u = np.zeros(prob.n_dof)
        u[lat.load_axis::prob.d] = prob.case.top_displacement(step) / lat.height * lat.X[:, lat.load_axis]
    else:
        u = 2 * u_prev - (0.0 if u_prev2 is None else u_prev2)
    g = prob.dirichlet_values(step)
    u[prob.fixed] = g[prob.fixed]
    return u


def newton_solve(prob, u0, tol=1e-8, max_it=50, mu=None, solver=None):
    """Newton iterations from u0 (Dirichlet values already in u0).  Returns (u, report)."""
    u = u0.copy()
    free = prob.free
    r = prob.residual(u, mu)
    rn = np.linalg.norm(r[free])
    r0 = rn
    hist, ls = [rn], []
    floor = 1e-12 * max(np.linalg.norm(r), 1e-300)
    it = 0
    while rn > tol * r0 and rn > floor and it < max_it:
        K = prob.tangent(u, mu)
        Kff = K[free][:, free].tocsc()
        if solver is None:
            du = spla.splu(Kff).solve(-r[free])
        else:
            du = solver(Kff, -r[free])
        m, accepted = 0, False
        while m <= MAX_M:
            step = BETA ** m
            ut = u.copy()
            ut[free] += step * du
            if prob.min_jacobian(ut) > 0:
                rt = prob.residual(ut, mu)
                rtn = np.linalg.norm(rt[free])
                if rtn <= (1 - C_ARMIJO * step) * rn:
                    accepted = True
                    break
            m += 1
        if not accepted:
            return u, NewtonReport(it, hist, ls, False)
        u, r, rn = ut, rt, rtn
        ls.append(m)
        hist.append(rn)
        floor = 1e-12 * max(np.linalg.norm(r), 1e-300)
        it += 1
    return u, NewtonReport(it, hist, ls, bool(rn <= tol * r0 or rn <= floor))


def load_path(prob, n_steps=None, tol=1e-8, max_it=50, mu=None, callback=None):
    """Run load steps 1..n_steps; returns the list of converged global displacements."""
    n_steps = prob.case.n_steps if n_steps is None else n_steps
    states, reports = [], []
    u1 = u2 = None
    for k in range(1, n_steps + 1):
        u0 = predictor(prob, k, u1, u2)
        u, rep = newton_solve(prob, u0, tol=tol, max_it=max_it, mu=mu)
        if not rep.converged:
            raise RuntimeError(f"oracle Newton failed at load step {k}")
        states.append(u)
        reports.append(rep)
        if callback is not None:
            callback(k, u, rep)
        u2, u1 = u1, u
    return states, reports


def compliance(prob, u, mu=None):
    """End compliance J = sum over Dirichlet DOFs of u_D f_D(u) (reaction work)."""
    r = prob.residual(u, mu)
    fixed = prob.fixed
    return float(np.dot(u[fixed], r[fixed]))
