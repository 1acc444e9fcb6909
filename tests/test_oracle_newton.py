"""Pins of the oracle's Newton solver, FETI-DP system and adjoint -- CPU."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import latgen
from oracle import adjoint, greedy, newton, rom
from oracle import cell as C
from oracle.assembly import Problem
from oracle.fetidp import FetiDP


def _block_case(d, dims, strain, theta=None):
    X, E = latgen.solid_cell(2, d)
    lat = latgen.tile(X, E, dims)
    th = np.ones(lat.n_cells) if theta is None else theta
    return latgen.LoadCase("block", lat, 1.0, 4.0, th, strain, 1, 1e-3)


@pytest.mark.parametrize("d", [2, 3])
def test_uniaxial_strain_block_solve(d):
    dims = (2, 2) if d == 2 else (1, 2, 2)
    case = _block_case(d, dims, 0.1)
    prob = Problem(case, lateral_rollers=True)
    u0 = newton.predictor(prob, 1, None, None)
    rng = np.random.default_rng(0)
    u0[prob.free] += 0.01 * rng.uniform(-1, 1, prob.free.size)
    u, rep = newton.newton_solve(prob, u0, tol=1e-12)
    assert rep.converged
    s = 1 - 0.1
    exact = np.zeros((prob.lat.n_nodes, d))
    exact[:, -1] = (s - 1) * prob.lat.X[:, -1]
    assert np.abs(u - exact.ravel()).max() < 1e-10
    # reaction work and its closed-form derivative w.r.t. a common shear-modulus factor
    H = prob.lat.height
    area = np.prod(dims[:-1])
    P = (s * s - 1) / s + 4.0 * np.log(s) / s
    J = newton.compliance(prob, u)
    assert abs(J - (s - 1) * H * P * area) < 1e-10
    g = adjoint.gradient(prob, u)
    assert abs(g.sum() - (s - 1) * H * area * (s * s - 1) / s) < 1e-10


def test_newton_quadratic_convergence():
    case = latgen.make_case("ring4")
    prob = Problem(case)
    u0 = newton.predictor(prob, 1, None, None)
    u, rep = newton.newton_solve(prob, u0, tol=1e-13)
    h = np.asarray(rep.residual_history) / rep.residual_history[0]
    assert rep.converged and rep.iterations <= 8
    # quadratic rate in the last steps: log r_{k+1} / log r_k close to 2
    k = int(np.argmax(h < 1e-3))
    assert k > 0 and k + 1 < len(h)
    assert np.log(h[k + 1]) / np.log(h[k]) > 1.7


@pytest.mark.parametrize("name", ["ring2", "strut2"])
def test_fetidp_saddle_point_equals_direct_solve(name):
    case = latgen.make_case(name)
    prob = Problem(case)
    u = newton.predictor(prob, 1, None, None)
    rng = np.random.default_rng(1)
    u[prob.free] += 0.002 * rng.uniform(-1, 1, prob.free.size)
    ul = prob.local(u)
    Kc = C.tangent(prob.cell, ul, prob.mu_cells, prob.lam)
    fc = C.internal_force(prob.cell, ul, prob.mu_cells, prob.lam).reshape(prob.lat.n_cells, -1)
    feti = FetiDP(prob)
    du, lam = feti.solve(Kc, fc)
    K = prob.tangent(u)
    r = prob.residual(u)
    free = prob.free
    ref = spla.spsolve(K[free][:, free].tocsc(), -r[free])
    assert np.abs(du[free] - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.all(du[prob.fixed] == 0)
    # the same with reduced local tangents: equals the assembled reduced system
    T = C.snapshots(prob.cell, ul, prob.mu_cells, prob.lam)
    g = greedy.greedy(T, 1e-3)
    al = greedy.alpha_triangular(T, g)
    Kt = rom.reduced_tangents(Kc[g.S], al)
    du2, _ = feti.solve(Kt, fc)
    A = rom.assembled(prob, Kt)
    ref2 = spla.spsolve(A[free][:, free].tocsc(), -r[free])
    assert np.abs(du2[free] - ref2).max() < 1e-9 * np.abs(ref2).max()


def test_adjoint_matches_finite_differences():
    case = latgen.make_case("ring2")
    prob = Problem(case)
    states, _ = newton.load_path(prob, tol=1e-13)
    u = states[-1]
    g = adjoint.gradient(prob, u)
    h = 1e-6
    base = prob.mu_cells.copy()
    for s in range(prob.lat.n_cells):
        Js = []
        for sign in (1, -1):
            mu = base.copy()
            mu[s] += sign * h * case.mu
            up, rep = newton.newton_solve(prob, u, tol=1e-13, mu=mu)
            assert rep.converged
            Js.append(newton.compliance(prob, up, mu))
        fd = (Js[0] - Js[1]) / (2 * h)
        assert abs(fd - g[s]) < 1e-6 * max(1.0, abs(g[s]))
