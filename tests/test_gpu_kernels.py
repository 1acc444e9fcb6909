"""GPU parity of the per-cell kernels, the greedy selection and the reduced tangent action.

Every comparison is element by element against the FP64 CPU oracle on the same seeded inputs.
Tolerances: FP64 paths agree to rounding (relative 1e-11 of the largest entry: the GPU sums in a
different order than numpy); the FP32 action to 2e-6 relative (24-bit mantissa, sums of a few
hundred terms).  Integer results (principal sets) must be identical.
"""
import numpy as np
import pytest
import torch

import latgen
from oracle import cell as OC
from oracle import greedy as OG
from oracle import newton as ON
from oracle import rom as OR
from oracle.assembly import Problem

pytestmark = pytest.mark.gpu

RTOL64 = 1e-11


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    from paper_2603_10741_gb300 import lattice
    return lattice


def _state(case, amp, seed):
    lat = case.lattice
    return latgen.smooth_state(lat, amp, seed).ravel()


def _rel(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name,amp", [("ring2", 0.01), ("ring4", 0.02), ("strut2", 0.01)])
def test_residual_and_tangent_parity(L, name, amp):
    case = latgen.make_case(name)
    prob = Problem(case)
    u = _state(case, amp, 11)
    lat = L.Lattice.from_case(case)
    ud = torch.tensor(u, device="cuda")
    out = lat.assemble_residual_tangent(ud, quad=0, residual=True, local_forces=True, tangent=True)
    r_ref = prob.residual(u)
    assert _rel(out["r"].cpu(), r_ref) < RTOL64
    f_ref = OC.internal_force(prob.cell, prob.local(u), prob.mu_cells, prob.lam)
    f_ref = f_ref.reshape(prob.lat.n_cells, -1).T
    assert _rel(out["f"].cpu(), f_ref) < RTOL64
    K_ref = OC.tangent(prob.cell, prob.local(u), prob.mu_cells, prob.lam)
    assert _rel(out["K"].cpu(), K_ref) < RTOL64
    assert abs(out["min_detF"] - OC.min_jacobian(prob.cell, prob.local(u)).min()) < 1e-12
    # reduced rule on a subset of cells (snapshot kernel)
    cells = np.array([prob.lat.n_cells - 1, 0], dtype=np.int32)
    red = lat.assemble_residual_tangent(ud, quad=1, cells=torch.tensor(cells, device="cuda"), residual=False,
                                        tangent=True)
    Kb_ref = OC.tangent(prob.cell, prob.local(u)[cells], prob.mu_cells[cells], prob.lam, reduced=True)
    assert _rel(red["K"].cpu(), Kb_ref) < RTOL64
    lat.close()


def test_gather_and_predictor_exact(L):
    case = latgen.make_case("ring4")
    prob = Problem(case)
    lat = L.Lattice.from_case(case)
    u = _state(case, 0.02, 3)
    x = lat.lattice_gather(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.array_equal(x, prob.local(u).reshape(prob.lat.n_cells, -1).T)
    u1 = lat.lattice_predictor(case.top_displacement(1)).cpu().numpy()
    assert np.array_equal(u1, ON.predictor(prob, 1, None, None))
    a = torch.tensor(_state(case, 0.01, 4), device="cuda")
    b = torch.tensor(_state(case, 0.01, 5), device="cuda")
    u3 = lat.lattice_predictor(case.top_displacement(3), a, b).cpu().numpy()
    assert np.abs(u3 - ON.predictor(prob, 3, a.cpu().numpy(), b.cpu().numpy())).max() < 1e-15
    lat.close()


def test_negative_jacobian_reported(L):
    case = latgen.make_case("ring2")
    lat = L.Lattice.from_case(case)
    u = np.zeros(lat.sizes.n_dof)
    u[0::2] = -3.0 * case.lattice.X[:, 0]          # folds every element: det F < 0
    with pytest.raises(L.LatticeError) as e:
        lat.assemble_residual_tangent(torch.tensor(u, device="cuda"))
    assert e.value.code == 4
    lat.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_greedy_parity_on_oracle_snapshots(L, seed):
    case = latgen.make_case("ring8")
    prob = Problem(case)
    u = _state(case, 0.03, 20 + seed)
    T = OC.snapshots(prob.cell, prob.local(u), prob.mu_cells, prob.lam)        # [nnz, N_s]
    eps = 1e-3
    g = OG.greedy(T, eps)
    a_ref = OG.alpha_triangular(T, g)
    lat = L.Lattice.from_case(case)
    out = lat.greedy_select(torch.tensor(T.T.copy(), device="cuda"), eps, 64)
    assert out["S"].cpu().numpy().tolist() == g.S.tolist()
    assert np.abs(out["max_res"] - np.asarray(g.max_res)).max() < 1e-12
    assert _rel(out["alpha"].cpu(), a_ref) < 1e-9
    assert _rel(out["beta"].cpu(), g.beta) < 1e-10
    assert _rel(out["Z"].cpu().T, g.Z) < 1e-10
    lat.close()


def test_greedy_degenerate_cases(L):
    lat = L.Lattice.from_case(latgen.make_case("ring2"))
    # identical columns up to scale: one principal, alpha = scale ratios
    rng = np.random.default_rng(4)
    t = rng.normal(size=40)
    sc = rng.uniform(0.5, 2.0, 7)
    T = np.outer(sc, t)                                   # [n_cols, n_rows]
    out = lat.greedy_select(torch.tensor(T, device="cuda"), 1e-10, 7)
    assert len(out["S"]) == 1
    s0 = int(out["S"][0])
    assert np.abs(out["alpha"].cpu().numpy()[0] - sc / sc[s0]).max() < 1e-12
    # orthogonal columns, ties broken to the lowest index, cap respected
    out = lat.greedy_select(torch.eye(5, dtype=torch.float64, device="cuda"), 0.1, 3)
    assert out["S"].cpu().tolist() == [0, 1, 2]
    lat.close()


def _select_and_reference(L, name, amp, seed, eps, precision=0):
    case = latgen.make_case(name)
    prob = Problem(case)
    u = _state(case, amp, seed)
    lat = L.Lattice.from_case(case, precision)
    sel = lat.select_principal_cells(torch.tensor(u, device="cuda"), eps, 128)
    T = OC.snapshots(prob.cell, prob.local(u), prob.mu_cells, prob.lam)
    g = OG.greedy(T, eps, 128)
    a_ref = OG.alpha_triangular(T, g)
    Kp_ref = OC.tangent(prob.cell, prob.local(u)[g.S], prob.mu_cells[g.S], prob.lam)
    return case, prob, lat, sel, g, a_ref, Kp_ref


def test_select_principal_cells_parity(L):
    case, prob, lat, sel, g, a_ref, Kp_ref = _select_and_reference(L, "ring8", 0.03, 7, 1e-3)
    assert sel["S"].cpu().numpy().tolist() == g.S.tolist()
    assert _rel(sel["alpha"].cpu(), a_ref) < 1e-9
    assert _rel(sel["Kp"].cpu(), Kp_ref) < RTOL64
    lat.close()


@pytest.mark.parametrize("name", ["ring8", "strut2"])
def test_reduced_apply_parity(L, name):
    case, prob, lat, sel, g, a_ref, Kp_ref = _select_and_reference(L, name, 0.02, 8, 1e-3)
    assert sel["S"].cpu().numpy().tolist() == g.S.tolist()
    s = lat.sizes
    X = latgen.uniform_field((s.n_loc, s.n_cells), 7)
    Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda")).cpu().numpy()
    Y_ref = OR.reduced_apply(prob.cell, Kp_ref, a_ref, X)
    assert _rel(Y, Y_ref) < 1e-10
    lat.close()
    # FP32 action from a mixed-precision handle
    case, prob, lat, sel, g, a_ref, Kp_ref = _select_and_reference(L, name, 0.02, 8, 1e-3, precision=1)
    Y32 = lat.apply_reduced_tangent(torch.tensor(X, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert _rel(Y32, Y_ref) < 2e-6
    lat.close()


def test_force_all_apply_is_per_cell(L):
    case = latgen.make_case("ring4")
    prob = Problem(case)
    u = _state(case, 0.02, 9)
    lat = L.Lattice.from_case(case)
    sel = lat.select_principal_cells(torch.tensor(u, device="cuda"), 0.0, 1, force_all=True)
    assert sel["n_r"] == prob.lat.n_cells
    K = OC.tangent(prob.cell, prob.local(u), prob.mu_cells, prob.lam)
    X = latgen.uniform_field((lat.sizes.n_loc, lat.sizes.n_cells), 7)
    Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda")).cpu().numpy()
    Y_ref = np.stack([prob.cell.dense(K[s]) @ X[:, s] for s in range(prob.lat.n_cells)], axis=1)
    assert _rel(Y, Y_ref) < RTOL64
    lat.close()


def _greedy_matches_oracle(prob, ul, eps, S, al):
    """Algorithm 1 run by the oracle on its own snapshot matrix of every cell (reduced rule at the
    same state): the same principal set in the same order, the same coefficients, and at the end
    of the oracle's trace the certified bound max_s ||Delta^s||_inf <= eps, unless the trace
    stopped at the cap of 256 principals."""
    T = OC.snapshots(prob.cell, ul, prob.mu_cells, prob.lam)
    g = OG.greedy(T, eps, 256)
    assert S.tolist() == g.S.tolist()
    al_ref = OG.alpha_triangular(T, g)
    assert np.abs(al - al_ref).max() <= 1e-9 * max(1.0, np.abs(al_ref).max())
    assert g.max_res[-1] <= eps or len(g.S) == 256


def test_full_size_ring32_sampled(L):
    """The 32x32 ring lattice (0.56 M DOF) at full size: residual, tangents and snapshots of 64
    seeded cells, the greedy on the full snapshot matrix and the apply on sampled cells."""
    case = latgen.make_case("ring32")
    prob = Problem(case)
    u = ON.predictor(prob, 2, None, None) + 0.002 * latgen.uniform_field(prob.n_dof, 13)
    u[prob.fixed] = ON.predictor(prob, 2, None, None)[prob.fixed]
    lat = L.Lattice.from_case(case)
    ud = torch.tensor(u, device="cuda")
    cells = np.sort(np.random.default_rng(14).choice(prob.lat.n_cells, 64, replace=False)).astype(np.int32)
    out = lat.assemble_residual_tangent(ud, local_forces=True, tangent=False)
    ul = prob.local(u)
    f_ref = OC.internal_force(prob.cell, ul[cells], prob.mu_cells[cells], prob.lam).reshape(64, -1).T
    assert _rel(out["f"].cpu().numpy()[:, cells], f_ref) < RTOL64
    ct = torch.tensor(cells, device="cuda")
    Kf = lat.assemble_residual_tangent(ud, quad=0, cells=ct, residual=False, tangent=True)["K"].cpu()
    assert _rel(Kf, OC.tangent(prob.cell, ul[cells], prob.mu_cells[cells], prob.lam)) < RTOL64
    sel = lat.select_principal_cells(ud, 3e-4, 256)
    assert 1 <= sel["n_r"] <= 256
    # the principal set is a valid greedy trace: every selected cell is principal with alpha = e_r
    al = sel["alpha"].cpu().numpy()
    S = sel["S"].cpu().numpy()
    assert np.abs(al[:, S] - np.eye(len(S))).max() < 1e-9
    _greedy_matches_oracle(prob, ul, 3e-4, S, al)
    Kp = sel["Kp"].cpu().numpy()
    assert _rel(Kp[:4], OC.tangent(prob.cell, ul[S[:4]], prob.mu_cells[S[:4]], prob.lam)) < RTOL64
    X = latgen.uniform_field((lat.sizes.n_loc, lat.sizes.n_cells), 7)
    Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda")).cpu().numpy()
    Y_ref = OR.reduced_apply(prob.cell, Kp, al[:, cells], X[:, cells])
    assert _rel(Y[:, cells], Y_ref) < 1e-10
    lat.close()


def test_full_size_strut10_sampled(L):
    """The 10x10x10 strut lattice (1.76 M DOF, 1000 cells of 880 nodes) at full size: residual
    forces and full-rule tangents of 32 seeded cells, the greedy on the full snapshot matrix, and
    the FP64 and FP32 reduced actions on sampled cells."""
    case = latgen.make_case("strut10")
    prob = Problem(case)
    u0 = ON.predictor(prob, 1, None, None)
    u = u0 + 0.001 * latgen.uniform_field(prob.n_dof, 17)
    u[prob.fixed] = u0[prob.fixed]
    lat = L.Lattice.from_case(case)
    ud = torch.tensor(u, device="cuda")
    cells = np.sort(np.random.default_rng(18).choice(prob.lat.n_cells, 32, replace=False)).astype(np.int32)
    out = lat.assemble_residual_tangent(ud, local_forces=True, tangent=False)
    ul = prob.local(u)
    f_ref = OC.internal_force(prob.cell, ul[cells], prob.mu_cells[cells], prob.lam).reshape(32, -1).T
    assert _rel(out["f"].cpu().numpy()[:, cells], f_ref) < RTOL64
    ct = torch.tensor(cells, device="cuda")
    Kf = lat.assemble_residual_tangent(ud, quad=0, cells=ct, residual=False, tangent=True)["K"].cpu()
    assert _rel(Kf, OC.tangent(prob.cell, ul[cells], prob.mu_cells[cells], prob.lam)) < RTOL64
    sel = lat.select_principal_cells(ud, 5e-3, 256)
    assert 1 <= sel["n_r"] <= 256
    al = sel["alpha"].cpu().numpy()
    S = sel["S"].cpu().numpy()
    assert np.abs(al[:, S] - np.eye(len(S))).max() < 1e-9
    _greedy_matches_oracle(prob, ul, 5e-3, S, al)
    Kp = sel["Kp"].cpu().numpy()
    assert _rel(Kp[:2], OC.tangent(prob.cell, ul[S[:2]], prob.mu_cells[S[:2]], prob.lam)) < RTOL64
    X = latgen.uniform_field((lat.sizes.n_loc, lat.sizes.n_cells), 19)
    Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda")).cpu().numpy()
    Y_ref = OR.reduced_apply(prob.cell, Kp, al[:, cells], X[:, cells])
    assert _rel(Y[:, cells], Y_ref) < 1e-10
    lat.close()
    # the FP32 action of a mixed-precision handle on the same state
    lat = L.Lattice.from_case(case, 1)
    sel32 = lat.select_principal_cells(ud, 5e-3, 256)
    assert sel32["S"].cpu().numpy().tolist() == S.tolist()
    Y32 = lat.apply_reduced_tangent(torch.tensor(X, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert _rel(Y32[:, cells], Y_ref) < 2e-6
    lat.close()


@pytest.mark.parametrize("name,n_r", [("ring8", 5), ("strut2", 3)])
def test_set_principal_cells_apply(L, name, n_r):
    """Caller-given principal cells and Dirichlet-distributed coefficients: the reduced action
    equals the oracle's sum_r alpha_r^s K^r x_s (FP64 exactly to rounding, FP32 to 2e-6)."""
    case = latgen.make_case(name)
    prob = Problem(case)
    u = _state(case, 0.02, 21)
    S = np.arange(n_r, dtype=np.int32)
    al = np.random.default_rng(8).dirichlet(np.ones(n_r), size=prob.lat.n_cells).T.copy()
    Kp = OC.tangent(prob.cell, prob.local(u)[S], prob.mu_cells[S], prob.lam)
    X = latgen.uniform_field((prob.cell.n_nodes * prob.cell.d, prob.lat.n_cells), 22)
    Y_ref = OR.reduced_apply(prob.cell, Kp, al, X)
    for prec, dt, tol in ((0, torch.float64, 1e-10), (1, torch.float32, 2e-6)):
        lat = L.Lattice.from_case(case, prec)
        lat.set_principal_cells(torch.tensor(u, device="cuda"), torch.tensor(S), torch.tensor(al))
        Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda", dtype=dt)).cpu().numpy()
        assert _rel(Y, Y_ref) < tol
        with pytest.raises(L.LatticeError):
            lat.set_principal_cells(torch.tensor(u, device="cuda"), torch.tensor([prob.lat.n_cells]),
                                    torch.ones((1, prob.lat.n_cells)))
        lat.close()


@pytest.mark.parametrize("dims", [(3, 1, 1), (2, 2, 1), (1, 1, 5)])
def test_apply_ragged_3d_cell_counts(L, dims):
    """3D strut lattices with 3, 4 and 5 cells: the FP32 action takes the node-group path only
    when the cell count is a multiple of four and the per-(cell, node) path otherwise; both must
    equal the oracle's sum_r alpha_r^s K^r x_s (caller-given principals and coefficients)."""
    Xr, E = latgen.strut_cell(6, 0.2)
    lat_geo = latgen.tile(Xr, E, dims)
    n = lat_geo.n_cells
    case = latgen.LoadCase(name="strut-ragged", lattice=lat_geo, mu=1.0, lam=4.0,
                           mu_scale=latgen.mu_scale(n, 9), total_strain=0.05, n_steps=5, eps=5e-3)
    prob = Problem(case)
    u = _state(case, 0.01, 23)
    n_r = min(2, n)
    S = np.arange(n_r, dtype=np.int32)
    al = latgen.dirichlet_coefficients(n_r, n, 8)
    Kp = OC.tangent(prob.cell, prob.local(u)[S], prob.mu_cells[S], prob.lam)
    X = latgen.uniform_field((prob.cell.n_nodes * 3, n), 24)
    Y_ref = OR.reduced_apply(prob.cell, Kp, al, X)
    for prec, dt, tol in ((0, torch.float64, 1e-10), (1, torch.float32, 2e-6)):
        lat = L.Lattice.from_case(case, prec)
        lat.set_principal_cells(torch.tensor(u, device="cuda"), torch.tensor(S), torch.tensor(al))
        Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda", dtype=dt)).cpu().numpy()
        assert _rel(Y, Y_ref) < tol
        lat.close()


@pytest.mark.parametrize("dims,n_r", [((5, 4, 7), 7), ((15, 14, 14), 1)])
def test_apply_node_groups(L, dims, n_r):
    """The FP32 node-group action on 12^3-voxel strut cells (2640 local DOF):
    140 cells (one full and one partial 128-cell tile) with 7 principals, whose blocks are staged
    in two chunks of shared memory (5 per chunk for the 8-node groups); and 2940 cells with one
    principal, which takes the 16-node groups (23 tiles x 55 groups >= 8 CTAs per SM on 152 SMs).
    Both equal the oracle's sum_r alpha_r^s K^r x_s on sampled cells, the partial tile's included;
    the FP64 action of the same handle pins the same cells to rounding."""
    Xr, E = latgen.strut_cell(12, 0.15)
    lat_geo = latgen.tile(Xr, E, dims)
    n = lat_geo.n_cells
    assert n % 4 == 0
    case = latgen.LoadCase(name="strut-groups", lattice=lat_geo, mu=1.0, lam=4.0,
                           mu_scale=latgen.mu_scale(n, 11), total_strain=0.05, n_steps=5, eps=5e-3)
    prob = Problem(case)
    u = _state(case, 0.01, 25)
    S = np.arange(n_r, dtype=np.int32) * 3
    al = latgen.dirichlet_coefficients(n_r, n, 12)
    Kp = OC.tangent(prob.cell, prob.local(u)[S], prob.mu_cells[S], prob.lam)
    X = latgen.uniform_field((prob.cell.n_nodes * 3, n), 26)
    rng = np.random.default_rng(27)
    cells = np.unique(np.concatenate([rng.choice(n, 40, replace=False), np.arange(n - 8, n), [0, 127, 128]]))
    Y_ref = OR.reduced_apply(prob.cell, Kp, al[:, cells], X[:, cells])
    for prec, dt, tol in ((0, torch.float64, 1e-10), (1, torch.float32, 2e-6)):
        lat = L.Lattice.from_case(case, prec)
        lat.set_principal_cells(torch.tensor(u, device="cuda"), torch.tensor(S), torch.tensor(al))
        Y = lat.apply_reduced_tangent(torch.tensor(X, device="cuda", dtype=dt)).cpu().numpy()
        assert _rel(Y[:, cells], Y_ref) < tol
        lat.close()


@pytest.mark.parametrize("name,eps", [("ring4", 1e-3), ("strut2", 1e-3), ("strut222", 5e-3)])
def test_dref_snapshot_selection_matches_oracle(L, name, eps):
    """Principal cells from D^ref snapshots (the pulled-back tangent tensor at the one-point
    rule, the Remark after Eq. snapshots): the same principal set, in the same order, and the same
    coefficients as the oracle's Algorithm 1 on its own D^ref snapshots of every cell."""
    case = latgen.make_case(name)
    prob = Problem(case)
    u = _state(case, 0.01, 23)
    ul = prob.local(u)
    T = OC.dref_snapshots(prob.cell, ul, prob.mu_cells, prob.lam)
    g = OG.greedy(T, eps, 256)
    al_ref = OG.alpha_triangular(T, g)
    lat = L.Lattice.from_case(case)
    lat.lattice_set_snapshots(1)
    sel = lat.select_principal_cells(torch.tensor(u, device="cuda"), eps, 256)
    assert sel["S"].cpu().numpy().tolist() == g.S.tolist()
    al = sel["alpha"].cpu().numpy()
    assert np.abs(al - al_ref).max() <= 1e-9 * max(1.0, np.abs(al_ref).max())
    lat.close()


def test_newton_with_dref_snapshots_ring4(L):
    """Three load steps of the 4x4 ring lattice with principal cells chosen on D^ref snapshots
    (FP64): the converged states are the oracle's (the snapshot kind changes the quasi-Newton
    operator, not the solution)."""
    from paper_2603_10741_gb300 import solve_load_path
    case = latgen.make_case("ring4")
    prob = Problem(case)
    ref, _ = ON.load_path(prob, n_steps=3, tol=1e-12)
    lat = L.Lattice.from_case(case)
    opts = lat.lattice_default_opts(newton_rtol=1e-12, snapshot=1)
    u, reps = solve_load_path(lat, case, opts, steps=3)
    err = np.linalg.norm(u.cpu().numpy() - ref[-1]) / np.linalg.norm(ref[-1])
    assert err < 1e-10, err
    lat.close()


def test_fp32_apply_on_unaligned_vectors(L):
    """The 3D FP32 action on cell vectors whose storage starts 4 bytes past a 16-byte boundary (a
    view into a larger buffer): the 16-byte staged kernel is not taken, the per-(cell, node)
    kernel gives the same result as on aligned vectors."""
    case = latgen.make_case("strut222")
    lat = L.Lattice.from_case(case, 1)
    s = lat.sizes
    u = lat.lattice_predictor(case.top_displacement(1))
    S = torch.arange(2, dtype=torch.int32)
    al = torch.tensor(latgen.dirichlet_coefficients(2, s.n_cells, 8))
    lat.set_principal_cells(u, S, al)
    n = s.n_loc * s.n_cells
    x = torch.tensor(latgen.uniform_field((s.n_loc, s.n_cells), 3), dtype=torch.float32, device="cuda")
    y = lat.apply_reduced_tangent(x)
    bx = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
    by = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
    xo = bx[1:n + 1].view(s.n_loc, s.n_cells)
    yo = by[1:n + 1].view(s.n_loc, s.n_cells)
    xo.copy_(x)
    assert xo.data_ptr() % 16 == 4
    lat.apply_reduced_tangent(xo, yo)
    assert _rel(yo.cpu().numpy(), y.cpu().numpy()) < 1e-6
    assert by[0].item() == 0.0 and by[n + 1].item() == 0.0   # nothing written outside the view
    lat.close()
