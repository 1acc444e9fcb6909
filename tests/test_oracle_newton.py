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


@pytest.mark.parametrize("name", ["ring2", "strut2"])
def test_load_predictor_reading(name):
    """The load-step predictor (reading of the paper's silent load stepping): step 1 is the affine
    field u_axis = (delta_1 / H) X_axis, step k >= 2 the extrapolation 2 u_{k-1} - u_{k-2} (u_0 = 0),
    then the Dirichlet values of step k: bottom face 0, top face -(k / n) strain H on the load axis
    and 0 across it.  Expected values are written node by node from the lattice coordinates."""
    case = latgen.make_case(name)
    prob = Problem(case)
    lat = prob.lat
    d, ax, H = lat.dim, lat.load_axis, lat.height
    n_steps, strain = case.n_steps, case.total_strain
    rng = np.random.default_rng(11)
    u1 = rng.uniform(-0.1, 0.1, prob.n_dof)
    u2 = rng.uniform(-0.1, 0.1, prob.n_dof)

    def expected(k, base):
        out = base.copy()
        delta = -(k / n_steps) * strain * H
        for node in range(lat.n_nodes):
            z = lat.X[node, ax]
            if abs(z) < 1e-12 or abs(z - H) < 1e-12:
                for i in range(d):
                    out[node * d + i] = delta if (abs(z - H) < 1e-12 and i == ax) else 0.0
        return out

    aff = np.zeros(prob.n_dof)
    for node in range(lat.n_nodes):
        aff[node * d + ax] = -(1 / n_steps) * strain * H / H * lat.X[node, ax]
    assert np.array_equal(newton.predictor(prob, 1, None, None), expected(1, aff))
    assert np.array_equal(newton.predictor(prob, 2, u1, None), expected(2, 2 * u1))
    assert np.allclose(newton.predictor(prob, 3, u1, u2), expected(3, 2 * u1 - u2), rtol=0, atol=1e-15)


def _strut_lattice(n, strain, steps):
    X, E = latgen.strut_cell(12, 0.15)
    lat = latgen.tile(X, E, (n, n, n))
    return latgen.LoadCase("strut", lat, 1.0, 4.0, np.ones(lat.n_cells), strain, steps, 5e-3)


def test_oracle_3d_strut_load_path_converges_symmetric():
    """The oracle's load path on a 2 x 2 x 2 lattice of the 12^3-voxel edge-strut cell: -1 % per
    step for three steps, each converging quadratically to 1e-10; with equal cells the solution
    keeps the lattice's symmetries (mirror x, mirror y, swap x <-> y), which a wrong index or sign
    in the 3D force, tangent or assembly would break."""
    case = _strut_lattice(2, 0.15, 15)
    prob = Problem(case)
    states, reps = newton.load_path(prob, n_steps=3, tol=1e-10)
    lat = prob.lat
    key = {tuple(np.round(x * 12).astype(int)): i for i, x in enumerate(lat.X)}
    maps = [(lambda x: (24 - x[0], x[1], x[2]), np.diag([-1, 1, 1])),
            (lambda x: (x[0], 24 - x[1], x[2]), np.diag([1, -1, 1])),
            (lambda x: (x[1], x[0], x[2]), np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]]))]
    for rep in reps:
        h = np.asarray(rep.residual_history) / rep.residual_history[0]
        assert rep.converged and rep.iterations <= 6
        assert h[-2] < 1e-3 and h[-1] < 1e-10
    for u in states:
        U = u.reshape(-1, 3)
        for f, Q in maps:
            img = np.array([key[f(tuple(np.round(x * 12).astype(int)))] for x in lat.X])
            assert np.abs(U[img] - U @ Q.T).max() < 1e-9 * np.abs(U).max()
    # the reaction grows with the compression (no softening within the first 3 %)
    react = [-prob.residual(u)[prob.top_axis_dofs].sum() for u in states]
    assert react[0] > 0 and react[1] > react[0] and react[2] > react[1]
