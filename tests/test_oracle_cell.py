"""Pins of the oracle's per-cell force and tangent (Eq. internalloadvec, Section 3.1.4) -- CPU."""
import numpy as np
import pytest

import latgen
from oracle import cell as C
from oracle.assembly import Problem


def _case(X, E, dims, mu=1.0, lam=4.0):
    lat = latgen.tile(X, E, dims)
    return latgen.LoadCase("t", lat, mu, lam, np.ones(lat.n_cells), 0.1, 1, 1e-3)


@pytest.mark.parametrize("which", ["ring", "strut"])
def test_rigid_motion_zero_residual(which):
    if which == "ring":
        case = _case(*latgen.ring_cell(8), (2, 2))
        R = np.array([[np.cos(0.7), -np.sin(0.7)], [np.sin(0.7), np.cos(0.7)]])
    else:
        case = _case(*latgen.strut_cell(6, 0.2), (2, 1, 1))
        a, b = 0.5, -0.9
        Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
        Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
        R = Rz @ Rx
    prob = Problem(case)
    X = prob.lat.X
    u = (X @ R.T - X + 0.3).ravel()
    assert np.abs(prob.residual(u)).max() < 1e-12


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("s", [0.9, 1.05])
def test_uniaxial_strain_patch_and_reaction(d, s):
    X, E = latgen.solid_cell(3, d)
    dims = (2, 3) if d == 2 else (2, 1, 2)
    prob = Problem(_case(X, E, dims))
    lat = prob.lat
    ax = lat.load_axis
    u = np.zeros((lat.n_nodes, d))
    u[:, ax] = (s - 1) * lat.X[:, ax]
    r = prob.residual(u.ravel()).reshape(-1, d)
    ext = np.asarray(lat.dims, dtype=float)
    boundary = np.any((np.abs(lat.X) < 1e-12) | (np.abs(lat.X - ext) < 1e-12), axis=1)
    assert np.abs(r[~boundary]).max() < 1e-13             # patch test: interior forces vanish
    P = 1.0 * (s * s - 1) / s + 4.0 * np.log(s) / s      # first Piola P_axis,axis = sigma_axis,axis
    area = np.prod([ext[k] for k in range(d) if k != ax])
    top = lat.top_nodes()
    assert abs(r[top, ax].sum() - P * area) < 1e-12 * max(1, abs(P))


def _linear_q1_stiffness(h, d, mu, lam):
    """Textbook B-matrix (Voigt) stiffness of an axis-aligned cube element of side h."""
    g = 1 / np.sqrt(3)
    nodes = latgen.solid_cell(1, d)[0] * 2 - 1                   # local node positions in [-1,1]^d
    pts = np.array(np.meshgrid(*[[-g, g]] * d, indexing="ij")).reshape(d, -1).T
    nv = 3 if d == 2 else 6
    Cv = np.zeros((nv, nv))
    Cv[:d, :d] = lam
    Cv[range(d), range(d)] += 2 * mu
    Cv[range(d, nv), range(d, nv)] = mu
    shear = [(0, 1)] if d == 2 else [(1, 2), (0, 2), (0, 1)]
    K = np.zeros((2 ** d * d, 2 ** d * d))
    for p in pts:
        Bm = np.zeros((nv, 2 ** d * d))
        for a, na in enumerate(nodes):
            grad = np.array([na[k] * np.prod([1 + na[m] * p[m] for m in range(d) if m != k])
                             for k in range(d)]) / 2 ** d * (2 / h)
            for k in range(d):
                Bm[k, a * d + k] = grad[k]
            for v, (i, j) in enumerate(shear):
                Bm[d + v, a * d + i] = grad[j]
                Bm[d + v, a * d + j] = grad[i]
        K += Bm.T @ Cv @ Bm * (h / 2) ** d
    return K


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_at_rest_is_linear_elastic(d):
    X, E = latgen.solid_cell(1, d)
    cell = C.RefCell(X * 0.5, E)          # one element of side 0.5
    K = cell.dense(C.tangent(cell, np.zeros((1, 2 ** d, d)), np.array([1.3]), 4.0)[0])
    ref = _linear_q1_stiffness(0.5, d, 1.3, 4.0)
    assert np.abs(K - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("which", ["ring", "strut"])
def test_tangent_central_difference_and_symmetry(which):
    X, E = latgen.ring_cell(4) if which == "ring" else latgen.strut_cell(4, 0.3)
    cell = C.RefCell(X, E)
    rng = np.random.default_rng(1)
    u = 0.01 * rng.uniform(-1, 1, (1, cell.n_nodes, cell.d))
    v = rng.uniform(-1, 1, (1, cell.n_nodes, cell.d))
    mu = np.array([1.1])
    K = cell.dense(C.tangent(cell, u, mu, 4.0)[0])
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    Kv = K @ v.ravel()
    errs = []
    for h in (1e-4, 5e-5):
        fd = (C.internal_force(cell, u + h * v, mu, 4.0) - C.internal_force(cell, u - h * v, mu, 4.0))
        errs.append(np.abs(fd.ravel() / (2 * h) - Kv).max())
    assert errs[1] < 1e-4 * np.abs(Kv).max()
    assert 3.5 < errs[0] / errs[1] < 4.5                   # O(h^2) central difference


def test_snapshot_is_reduced_rule_tangent():
    X, E = latgen.ring_cell(4)
    cell = C.RefCell(X, E)
    rng = np.random.default_rng(2)
    u = 0.02 * rng.uniform(-1, 1, (3, cell.n_nodes, 2))
    T = C.snapshots(cell, u, np.ones(3), 4.0)
    assert T.shape == (cell.nnz, 3)
    # one-point rule: the element matrix is the centre-point integrand times the element area
    Kbar = C.tangent(cell, u, np.ones(3), 4.0, reduced=True)
    assert np.array_equal(T, Kbar.T)
    # the one-point rule itself is pinned to a closed form below


def test_pattern_covers_element_pairs():
    X, E = latgen.ring_cell(8)
    cell = C.RefCell(X, E)
    assert cell.nnz == 2496
    X, E = latgen.ring_cell(16)
    assert C.RefCell(X, E).nnz == 9600


def _q1_corners(d):
    """Q1 node positions xi_a in [-1,1]^d: counter-clockwise, bottom face then top face."""
    sq = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
    if d == 2:
        return np.array(sq, dtype=float)
    return np.array([p + (z,) for z in (-1, 1) for p in sq], dtype=float)


def _one_point_stiffness(A, d, mu, lam):
    """Linear-elastic Q1 stiffness of the affine element X = X0 + A xi integrated with the single
    centre point (weight 2^d on [-1,1]^d): K = 2^d |det A| B(0)^T C B(0), with Voigt B(0) built
    from the centre gradients grad_xi phi_a(0) = xi_a / 2^d mapped by A^{-T}."""
    nodes = _q1_corners(d)
    Ainv_T = np.linalg.inv(A).T
    nv = 3 if d == 2 else 6
    Cv = np.zeros((nv, nv))
    Cv[:d, :d] = lam
    Cv[range(d), range(d)] += 2 * mu
    Cv[range(d, nv), range(d, nv)] = mu
    shear = [(0, 1)] if d == 2 else [(1, 2), (0, 2), (0, 1)]
    B = np.zeros((nv, 2 ** d * d))
    for a, xa in enumerate(nodes):
        g = Ainv_T @ (xa / 2 ** d)
        for k in range(d):
            B[k, a * d + k] = g[k]
        for v, (i, j) in enumerate(shear):
            B[d + v, a * d + i] = g[j]
            B[d + v, a * d + j] = g[i]
    return 2 ** d * abs(np.linalg.det(A)) * B.T @ Cv @ B


@pytest.mark.parametrize("d", [2, 3])
def test_one_point_rule_matches_closed_form_on_a_skewed_element(d):
    """Eq. (snapshots) with the one-point rule: at rest, the reduced-rule tangent of a skewed
    (affine, non-rectangular) element equals the hand-written centre-point stiffness; the
    full 2^d rule differs from it (the hourglass modes are stiff there)."""
    A = np.array([[0.5, 0.15], [0.05, 0.4]]) if d == 2 else \
        np.array([[0.5, 0.1, 0.05], [0.02, 0.45, 0.1], [0.08, 0.03, 0.4]]) / 2
    X = 0.3 + _q1_corners(d) @ A.T           # element node positions X_a = X0 + A xi_a
    E = np.arange(2 ** d)[None, :]
    cell = C.RefCell(X, E)
    zero = np.zeros((1, 2 ** d, d))
    K1 = cell.dense(C.tangent(cell, zero, np.array([1.3]), 4.0, reduced=True)[0])
    ref = _one_point_stiffness(A, d, 1.3, 4.0)
    assert np.abs(K1 - ref).max() < 1e-13 * np.abs(ref).max()
    K2 = cell.dense(C.tangent(cell, zero, np.array([1.3]), 4.0)[0])
    assert np.abs(K2 - ref).max() > 1e-2 * np.abs(ref).max()
    # one point sees only the centre strain: the rank is the number of strain components
    assert np.linalg.matrix_rank(K1, tol=1e-10 * np.abs(K1).max()) == (3 if d == 2 else 6)


@pytest.mark.parametrize("which", ["ring", "strut"])
def test_dref_snapshot_reassembles_the_reduced_rule_tangent(which):
    """The D^ref snapshot (pulled-back tangent tensor at the one-point rule, Eq.
    tensorfunctionPulledback) contracted with the reference gradients of the Q1 element at its
    centre, times the one-point weight 2^d, gives back the reduced-rule tangent computed through
    the current-configuration gradients (Eq. stiffmatPulledback): a check of the pull-back's
    index placement and Jacobian factor against an independent path."""
    X, E = latgen.ring_cell(4) if which == "ring" else latgen.strut_cell(4, 0.3)
    cell = C.RefCell(X, E)
    d = cell.d
    rng = np.random.default_rng(7)
    u = 0.02 * rng.uniform(-1, 1, (2, cell.n_nodes, d))
    mu = np.array([1.1, 0.9])
    T = C.dref_snapshots(cell, u, mu, 4.0)
    assert T.shape == (cell.n_el * d ** 4, 2)
    Kbar = C.tangent(cell, u, mu, 4.0, reduced=True)
    corners = _q1_corners(d)
    g0 = corners / 2 ** d                                  # dphi_a / dxi at the element centre
    for s in range(2):
        Dref = T[:, s].reshape(cell.n_el, d, d, d, d)
        K = np.zeros((cell.n_nodes * d, cell.n_nodes * d))
        for e, el in enumerate(cell.elems):
            Ke = 2 ** d * np.einsum("ijmn,am,bn->aibj", Dref[e], g0, g0)
            for a, na in enumerate(el):
                for b, nb in enumerate(el):
                    K[na * d:(na + 1) * d, nb * d:(nb + 1) * d] += Ke[a, :, b, :]
        ref = cell.dense(Kbar[s])
        assert np.abs(K - ref).max() < 1e-12 * np.abs(ref).max()


def test_dref_snapshot_at_rest_is_the_pulled_back_elasticity():
    """At rest on an axis-aligned element of side h (J = (h/2) I): D^ref_ijmn = C_imjn (2/h)^2
    (h/2)^d with C_ikjl = lam d_ik d_jl + mu (d_ij d_kl + d_il d_kj) (no stress, J = 1)."""
    d, h, mu, lam = 3, 0.5, 1.3, 4.0
    X, E = latgen.solid_cell(1, d)
    cell = C.RefCell(X * h, np.asarray(E))
    T = C.dref_snapshots(cell, np.zeros((1, cell.n_nodes, d)), np.array([mu]), lam)
    Dref = T[:, 0].reshape(d, d, d, d)
    dl = np.eye(d)
    ref = np.zeros((d, d, d, d))
    for i in range(d):
        for j in range(d):
            for m in range(d):
                for n in range(d):
                    ref[i, j, m, n] = lam * dl[i, m] * dl[j, n] + mu * (dl[i, j] * dl[m, n] + dl[i, n] * dl[m, j])
    ref *= (2 / h) ** 2 * (h / 2) ** d
    assert np.abs(Dref - ref).max() < 1e-13 * np.abs(ref).max()
