"""GPU parity of the FETI-DP pieces, the Krylov solve, Newton load stepping and the adjoint.

The reference is the FP64 CPU oracle: direct sparse solves of the assembled system (exact
tangent, or the reduced tangents sum_r alpha_r^s K^r of the oracle's own greedy), Newton with
Armijo backtracking, and the direct adjoint.  Tolerances follow from the solver tolerances:
the Krylov relative residual 1e-12 gives directions within ~1e-9; Newton solutions converged to
1e-12 agree to 1e-10 relative L2 (FP64 mode); in the mixed modes only the preconditioner is
FP32 (the Krylov operator, residual and update stay FP64), so the solution converges to the
Newton tolerance (1e-8 relative residual) of the oracle's solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import latgen
from oracle import adjoint as OA
from oracle import cell as OC
from oracle import greedy as OG
from oracle import newton as ON
from oracle import rom as OR
from oracle.assembly import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    from paper_2603_10741_gb300 import lattice
    return lattice


def _u0(prob, step=1, jitter=0.0, seed=0):
    u = ON.predictor(prob, step, None, None)
    if jitter:
        rng = np.random.default_rng(seed)
        u[prob.free] += jitter * rng.uniform(-1, 1, prob.free.size)
    return u


def test_jump_of_continuous_vector_is_zero_and_roundtrip(L):
    case = latgen.make_case("strut2")
    prob = Problem(case)
    lat = L.Lattice.from_case(case)
    u = latgen.smooth_state(case.lattice, 0.01, 1).ravel()
    u[prob.fixed] = 0
    ud = torch.tensor(u, device="cuda")
    lat.select_principal_cells(ud, 1e-3)
    lat.lattice_prepare_solver(ud)
    v = lat.feti_from_global(ud)
    s = lat.sizes
    w = lat.feti_apply(0, v).cpu().numpy()
    lam = w[s.n_loc * s.n_cells + s.n_primal:]
    assert lam.size == s.n_lambda and np.abs(lam).max() < 1e-15
    back = lat.feti_to_global(v).cpu().numpy()
    assert np.abs(back - u).max() < 1e-15
    lat.close()


@pytest.mark.parametrize("name", ["ring4", "strut2"])
def test_force_all_local_inverse_is_exact(L, name):
    """With every cell principal, K^-rom is the exact partially assembled inverse (Section 3.3.1)."""
    case = latgen.make_case(name)
    prob = Problem(case)
    lat = L.Lattice.from_case(case)
    ud = torch.tensor(_u0(prob, 1, 0.002, 1), device="cuda")
    lat.select_principal_cells(ud, 0.0, 1, force_all=True)
    # the local blocks from the full tangent (the material-part option builds them from another
    # matrix, so it gives a preconditioner, not the inverse of K~)
    lat.lattice_prepare_solver(ud, lat.lattice_default_opts(precond_tangent=0))
    s = lat.sizes
    rng = np.random.default_rng(3)
    v = lat.feti_from_global(torch.tensor(rng.uniform(-1, 1, s.n_dof), device="cuda"))
    # remove the multiplier part, apply K~ then K^-rom
    v[s.n_loc * s.n_cells + s.n_primal:] = 0
    Kv = lat.feti_apply(0, v)
    Kv[s.n_loc * s.n_cells + s.n_primal:] = 0
    back = lat.feti_apply(1, Kv)
    nd = s.n_loc * s.n_cells + s.n_primal
    err = (back[:nd] - v[:nd]).abs().max().item() / v[:nd].abs().max().item()
    assert err < 1e-9
    lat.close()


@pytest.mark.parametrize("force_all", [True, False])
@pytest.mark.parametrize("name,strain,pre", [("ring4", 0.01, -1), ("strut2", 0.002, 0), ("strut2", 0.002, 1),
                                             ("strut2", 0.01, 1)])
def test_krylov_solve_matches_direct_solve(L, name, strain, pre, force_all):
    """The FGMRES solution on the FETI-DP saddle point equals the oracle's direct solve of the
    assembled (exact, or reduced sum_r alpha_r^s K^r) tangent system for the Newton rhs -r.
    On the strut cells at 0.2 % compression the corner-only local blocks of the full tangent are
    still definite; at 1 % they are not, and the preconditioner is built from the material part
    of the principal tangents (pre = 1), which does not change the solution."""
    case = latgen.make_case(name)
    case.total_strain = strain
    prob = Problem(case)
    u0 = _u0(prob, 1, 0.0005 if name == "ring4" else 0.0001, 2)
    lat = L.Lattice.from_case(case)
    eps = 1e-3
    opts = lat.lattice_default_opts(eps=eps, force_all=int(force_all), krylov_rtol=1e-12, krylov_max_it=3000,
                                    precond_tangent=pre)
    ud = torch.tensor(u0, device="cuda")
    sel = lat.select_principal_cells(ud, eps, 256, force_all=force_all)
    lat.lattice_prepare_solver(ud, opts)
    r = prob.residual(u0)
    x, its, rel = lat.tangent_solve(torch.tensor(-r, device="cuda"), opts)
    assert rel <= 1e-12
    x = x.cpu().numpy()
    free = prob.free
    if force_all:
        A = prob.tangent(u0)
    else:
        ul = prob.local(u0)
        T = OC.snapshots(prob.cell, ul, prob.mu_cells, prob.lam)
        g = OG.greedy(T, eps, 256)
        assert sel["S"].cpu().numpy().tolist() == g.S.tolist()
        al = OG.alpha_triangular(T, g)
        Kp = OC.tangent(prob.cell, ul[g.S], prob.mu_cells[g.S], prob.lam)
        A = OR.assembled(prob, OR.reduced_tangents(Kp, al))
    ref = spla.spsolve(A[free][:, free].tocsc(), -r[free])
    assert np.abs(x[free] - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.all(x[prob.fixed] == 0)
    lat.close()


@pytest.mark.parametrize("force_all", [True, False])
def test_newton_load_path_ring4_fp64(L, force_all):
    """The 4x4 ring lattice, 8x8 Q1 per cell, -10 % in 10 steps: the GPU load path (plain full
    tangent or reduced basis, FP64) reaches the oracle's solution at every step."""
    from paper_2603_10741_gb300 import solve_load_path
    case = latgen.make_case("ring4")
    prob = Problem(case)
    ref, ref_reps = ON.load_path(prob, tol=1e-12)
    lat = L.Lattice.from_case(case)
    opts = lat.lattice_default_opts(newton_rtol=1e-12, force_all=int(force_all), krylov_rtol=1e-12)
    states = []
    u, reps = solve_load_path(lat, case, opts, log=lambda k, rep: None)
    got = u.cpu().numpy()
    err = np.linalg.norm(got - ref[-1]) / np.linalg.norm(ref[-1])
    assert err < 1e-10, err
    its = sum(r["iterations"] for r in reps)
    its_ref = sum(r.iterations for r in ref_reps)
    if force_all:
        assert its <= its_ref + 2              # exact Newton, same iteration counts
    else:
        assert its <= 4 * its_ref              # quasi-Newton with the reduced tangent
    lat.close()


@pytest.mark.parametrize("precision", [1])
def test_newton_mixed_precision_ring4(L, precision):
    case = latgen.make_case("ring4")
    prob = Problem(case)
    ref, _ = ON.load_path(prob, n_steps=3, tol=1e-12)
    from paper_2603_10741_gb300 import solve_load_path
    lat = L.Lattice.from_case(case, precision)
    opts = lat.lattice_default_opts(newton_rtol=1e-10)
    u, reps = solve_load_path(lat, case, opts, steps=3)
    got = u.cpu().numpy()
    err = np.linalg.norm(got - ref[-1]) / np.linalg.norm(ref[-1])
    assert err < 1e-8, err
    r = prob.residual(got)
    r0 = prob.residual(ON.predictor(prob, 3, ref[1], ref[0]))
    assert np.linalg.norm(r[prob.free]) <= 1e-8 * np.linalg.norm(r0[prob.free])
    lat.close()


def test_adjoint_gradient_matches_oracle(L):
    case = latgen.make_case("ring2")
    prob = Problem(case)
    states, _ = ON.load_path(prob, tol=1e-13)
    u = states[-1]
    g_ref = OA.gradient(prob, u)
    J_ref = ON.compliance(prob, u)
    lat = L.Lattice.from_case(case)
    opts = lat.lattice_default_opts(eps=1e-4)
    g, J, rep = lat.adjoint_gradient(torch.tensor(u, device="cuda"), opts)
    assert rep.converged
    assert abs(J - J_ref) < 1e-12 * abs(J_ref)
    assert np.abs(g.cpu().numpy() - g_ref).max() < 1e-9 * np.abs(g_ref).max()
    lat.close()


def test_checkpoint_roundtrip(L, tmp_path):
    case = latgen.make_case("ring2")
    lat = L.Lattice.from_case(case)
    a = torch.rand(lat.sizes.n_dof, dtype=torch.float64, device="cuda")
    b = torch.rand(lat.sizes.n_dof, dtype=torch.float64, device="cuda")
    lat.lattice_checkpoint_save(tmp_path / "c.ckpt", 3, -0.25, a, b)
    step, load, a2, b2 = lat.lattice_checkpoint_load(tmp_path / "c.ckpt")
    assert step == 3 and load == -0.25
    assert torch.equal(a, a2) and torch.equal(b, b2)
    lat.close()


@pytest.mark.parametrize("name", ["ring8"])
def test_bf16_tensor_core_local_product(L, name):
    """BF16 mode: the tcgen05 principal-block product inside K^-rom agrees with the FP64 one to
    the accuracy of its BF16 operand pairs (~16-bit mantissas; the dropped low x low product is
    ~2^-16 relative) with FP32 accumulation over ~570 terms."""
    case = latgen.make_case(name)
    prob = Problem(case)
    ud = torch.tensor(_u0(prob, 1, 0.0005, 4), device="cuda")
    outs = []
    for prec in (0, 2):
        lat = L.Lattice.from_case(case, prec)
        opts = lat.lattice_default_opts(eps=1e-3)
        lat.select_principal_cells(ud, 1e-3, 256)
        lat.lattice_prepare_solver(ud, opts)
        s = lat.sizes
        rng = np.random.default_rng(5)
        v = lat.feti_from_global(torch.tensor(rng.uniform(-1, 1, s.n_dof), device="cuda"))
        outs.append(lat.feti_apply(1, v)[: s.n_loc * s.n_cells + s.n_primal].cpu().numpy())
        lat.close()
    ref, got = outs
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err


def test_newton_bf16_mode_ring4(L):
    """BF16 preconditioner blocks, FP64 residual/operator/update: same solution as the oracle."""
    from paper_2603_10741_gb300 import solve_load_path
    case = latgen.make_case("ring4")
    prob = Problem(case)
    ref, _ = ON.load_path(prob, n_steps=2, tol=1e-12)
    lat = L.Lattice.from_case(case, 2)
    u, reps = solve_load_path(lat, case, lat.lattice_default_opts(newton_rtol=1e-10), steps=2)
    err = np.linalg.norm(u.cpu().numpy() - ref[-1]) / np.linalg.norm(ref[-1])
    assert err < 1e-8, err
    lat.close()


def test_tolerance_tightening_on_slow_reduced_newton(L):
    """ring4, FP64, three load steps from a greedy tolerance of 0.05 (one principal cell: the
    first greedy residual is 0.115 and all cells share one snapshot at the affine predictor),
    with eps_refine = 3 and a contraction test of 1e-3 (two steps in a row that reduce the
    residual by less than 1000x count as slow): eps is divided by 10 at least once, every
    report's eps_last is 0.05 10^-k for its k tightenings, and the load path still reaches the
    oracle's solution.  With eps_refine = 0 eps stays at 0.05."""
    from paper_2603_10741_gb300 import solve_load_path
    from paper_2603_10741_gb300.lattice import LatticeError
    case = latgen.make_case("ring4")
    prob = Problem(case)
    ref, _ = ON.load_path(prob, n_steps=3, tol=1e-12)
    for refine in (3, 0):
        lat = L.Lattice.from_case(case)
        opts = lat.lattice_default_opts(newton_rtol=1e-11, krylov_rtol=1e-12, eps=0.05, eps_refine=refine,
                                        eps_refine_rate=1e-3, newton_max_it=100)
        try:
            u, reps = solve_load_path(lat, case, opts, steps=3)
        except (LatticeError, RuntimeError):
            assert refine == 0                 # a rejected direction ends the call when eps is fixed
            lat.close()
            continue
        err = np.linalg.norm(u.cpu().numpy() - ref[-1]) / np.linalg.norm(ref[-1])
        assert err < 1e-9, (refine, err)
        for r in reps:
            assert r["eps_refinements"] <= refine
            assert abs(r["eps_last"] - 0.05 * 10.0 ** -r["eps_refinements"]) < 1e-12 * 0.05, r
        if refine:
            assert sum(r["eps_refinements"] for r in reps) >= 1, reps
        lat.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_blocked_coarse_inverse_matches_dense(L, precision):
    """Coarse solves on the 8x8 ring lattice: the block-LU sweeps over the cell layers (one
    16-CTA cluster per sweep with prefetched rows; one 8-CTA cluster reading rows from global
    memory; one whole-GPU launch per step; the whole solve as one cooperative launch) and the
    block-tridiagonal explicit
    inverse equal the dense inverse of the unlayered coarse matrix, and
    with every cell principal K^-rom stays the exact inverse of K~ in FP64.  In the FP32 mode
    (FP32 local inverses; the block-LU solve stays FP64, the explicit inverse is applied as an FP32
    copy) the three agree to FP32 rounding."""
    case = latgen.make_case("ring8")
    prob = Problem(case)
    ud = torch.tensor(_u0(prob, 1, 0.0005, 6), device="cuda")
    arrays = L.case_arrays(case)
    outs = []
    tol = 1e-9 if precision == 0 else 1e-5
    for layered, block_lu in ((True, 1), (True, 2), (True, 3), (True, 4), (True, 0), (False, 0)):
        a = dict(arrays)
        if not layered:
            a["cell_layer"] = None
        lat = L.Lattice(a, precision)
        lat.select_principal_cells(ud, 0.0, 1, force_all=True)
        lat.lattice_prepare_solver(ud, lat.lattice_default_opts(coarse_block_lu=block_lu))
        s = lat.sizes
        assert s.coarse_block_lu == (1 if layered and block_lu else 0)   # 2: block LU, full-GPU steps
        if layered:
            assert s.n_coarse_blocks >= 2 and s.coarse_block > 0
        rng = np.random.default_rng(7)
        v = lat.feti_from_global(torch.tensor(rng.uniform(-1, 1, s.n_dof), device="cuda"))
        nd = s.n_loc * s.n_cells + s.n_primal
        v[nd:] = 0
        Kv = lat.feti_apply(0, v)
        Kv[nd:] = 0
        back = lat.feti_apply(1, Kv)
        err = (back[:nd] - v[:nd]).abs().max().item() / v[:nd].abs().max().item()
        if precision == 0:
            assert err < 1e-9, (layered, block_lu, err)
        outs.append(back[:nd].cpu().numpy())
        lat.close()
    ref = np.abs(outs[5]).max()
    for k in range(4):
        assert np.abs(outs[k] - outs[5]).max() < tol * ref, k
    assert np.abs(outs[3] - outs[4]).max() < (1e-10 if precision == 0 else tol) * ref


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_newton_ring32_full_size_oracle_residual(L, precision):
    """The 32x32 ring lattice (556 034 DOF) at full size, in the configuration the benchmark
    times: one load step from the predictor with the reduced path (FP64, FP32 or BF16
    preconditioner).  The oracle's own residual at the GPU solution must meet the Newton
    tolerance (1e-8) relative to its residual at the predictor (rounding of the two residual
    evaluations is ~1e-11 of it), and the Dirichlet values must be untouched."""
    case = latgen.make_case("ring32")
    prob = Problem(case)
    lat = L.Lattice.from_case(case, precision)
    u0 = lat.lattice_predictor(case.top_displacement(1))
    u = u0.clone()
    opts = lat.lattice_default_opts(newton_rtol=1e-8)
    rep = lat.newton_step(u, opts)
    assert rep.converged and rep.n_r_last >= 1
    got = u.cpu().numpy()
    r = prob.residual(got)
    r0 = prob.residual(u0.cpu().numpy())
    ratio = np.linalg.norm(r[prob.free]) / np.linalg.norm(r0[prob.free])
    assert ratio <= 1.01e-8, ratio
    # Dirichlet values exactly as prescribed
    assert np.array_equal(got[prob.fixed], u0.cpu().numpy()[prob.fixed])
    lat.close()


def test_bf16_tensor_core_long_segments(L):
    """BF16 mode with few keys (at most three principals: eps 5e-2) on the 32x32 ring lattice, so
    that the key segments hold >= 96 cells on average (many full 64-cell tiles per key, as on
    the 3D lattices); the tensor-core product must agree with the FP64 one to the accuracy of
    the BF16 pairs."""
    case = latgen.make_case("ring32")
    prob = Problem(case)
    ud = torch.tensor(_u0(prob, 1, 0.0005, 4), device="cuda")
    outs = []
    for prec in (0, 2):
        lat = L.Lattice.from_case(case, prec)
        opts = lat.lattice_default_opts(eps=5e-2, max_enrich=0)
        sel = lat.select_principal_cells(ud, 5e-2, 256)
        assert 1 <= sel["n_r"] <= 3, sel["n_r"]
        lat.lattice_prepare_solver(ud, opts)
        s = lat.sizes
        rng = np.random.default_rng(6)
        v = lat.feti_from_global(torch.tensor(rng.uniform(-1, 1, s.n_dof), device="cuda"))
        outs.append(lat.feti_apply(1, v)[: s.n_loc * s.n_cells + s.n_primal].cpu().numpy())
        lat.close()
    ref, got = outs
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_error_against_oracle_by_precision(L, precision, capsys):
    """The errors of the displacements (4x4 ring lattice, three load steps) and of the adjoint
    gradient (2x2 ring lattice, end state) against the FP64 oracle, in each precision mode: FP64
    within 1e-10 (relative L2), the mixed modes within the Newton tolerance 1e-8; the gradient's
    defect correction uses the exact FP64 tangent action in every mode, so it stays within 1e-9
    of the oracle's.  The errors are printed for the record."""
    from paper_2603_10741_gb300 import solve_load_path
    case = latgen.make_case("ring4")
    prob = Problem(case)
    ref, _ = ON.load_path(prob, n_steps=3, tol=1e-13)
    lat = L.Lattice.from_case(case, precision)
    rtol = 1e-12 if precision == 0 else 1e-10
    u, _ = solve_load_path(lat, case, lat.lattice_default_opts(newton_rtol=rtol), steps=3)
    err_u = np.linalg.norm(u.cpu().numpy() - ref[-1]) / np.linalg.norm(ref[-1])
    lat.close()
    case2 = latgen.make_case("ring2")
    prob2 = Problem(case2)
    states, _ = ON.load_path(prob2, tol=1e-13)
    g_ref = OA.gradient(prob2, states[-1])
    lat = L.Lattice.from_case(case2, precision)
    g, J, rep = lat.adjoint_gradient(torch.tensor(states[-1], device="cuda"), lat.lattice_default_opts(eps=1e-4))
    err_g = np.abs(g.cpu().numpy() - g_ref).max() / np.abs(g_ref).max()
    lat.close()
    with capsys.disabled():
        print(f"\n[precision {precision}] displacement rel L2 error {err_u:.2e}, gradient max rel error {err_g:.2e}")
    assert err_u < (1e-10 if precision == 0 else 1e-8), err_u
    assert err_g < 1e-9, err_g


def test_bf16_tensor_core_3d_blocks(L):
    """The 10x10x10 strut lattice (n_R 2616: 41 K panels per pass, 21 row tiles; three keys of
    ~100-800 cells): the tensor-core product on the 3D blocks must agree with the FP64 product
    to the accuracy of the BF16 pairs."""
    case = latgen.make_case("strut10")
    outs = []
    for prec in (0, 2):
        lat = L.Lattice.from_case(case, prec)
        u = lat.lattice_predictor(case.top_displacement(1))
        opts = lat.lattice_default_opts(max_enrich=0)
        lat.select_principal_cells(u, opts.eps, 256)
        lat.lattice_prepare_solver(u, opts)
        s = lat.sizes
        rng = np.random.default_rng(7)
        v = lat.feti_from_global(torch.tensor(rng.uniform(-1, 1, s.n_dof), device="cuda"))
        outs.append(lat.feti_apply(1, v)[: s.n_loc * s.n_cells + s.n_primal].cpu().numpy())
        lat.close()
    ref, got = outs
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err


def _oracle_kinv_rom(prob, ul, eps, v_glob):
    """The oracle's reading of K^-rom (Section 3.3.1 with the principal-cell ROM of the local DD
    operators): the oracle's greedy on its own snapshots picks the principals; every cell s is
    tied to the principal r(s) whose snapshot is nearest in direction (largest cosine) with the
    scale c_s = |t^s| cos / |t^r(s)|; K^-rom is then the exact inverse of the partially assembled
    matrix built from the per-cell matrices c_s K^r(s) (corners primal), applied by a direct
    sparse solve to the saddle-point image of the global vector v_glob.  Returns the solution on
    the remaining (R) unknowns as {(cell, local dof): value}, and the FETI index sets."""
    import scipy.sparse as sp
    from oracle.fetidp import FetiDP
    T = OC.snapshots(prob.cell, ul, prob.mu_cells, prob.lam)
    g = OG.greedy(T, eps, 256)
    nrm = np.linalg.norm(T, axis=0)
    cosv = (T[:, g.S].T @ T) / (nrm[g.S][:, None] * nrm[None, :])       # [N_r, N_s]
    r_of = np.argmax(cosv, axis=0)
    c = nrm * cosv[r_of, np.arange(T.shape[1])] / nrm[g.S][r_of]
    Kp = OC.tangent(prob.cell, ul[g.S], prob.mu_cells[g.S], prob.lam)
    Khat = c[:, None] * Kp[r_of]
    fe = FetiDP(prob)
    idx = fe._index()
    n = fe.n_r + fe.n_p
    cell = prob.cell
    ri, ci = idx[:, cell.rows], idx[:, cell.cols]
    keep = (ri >= 0) & (ci >= 0)
    Kt = sp.csr_matrix((Khat[keep], (ri[keep], ci[keep])), shape=(n, n)).tocsc()
    rhs = np.zeros(n)
    cd = prob.cell_dofs
    ok = idx >= 0
    rhs[idx[ok]] = v_glob[cd[ok]]          # every copy (remaining) and each primal DOF once
    x = sp.linalg.spsolve(Kt, rhs)
    return x, idx, fe, len(g.S)


def test_bf16_tensor_core_kinv_matches_oracle_elementwise(L):
    """BF16 mode on the 8x8 ring lattice with few principals (eps 1e-2: the key segments are long
    enough for the tcgen05 product): K^-rom applied to the saddle-point image of a seeded global
    vector, element by element on every remaining local DOF, against the oracle's direct solve of
    the same ROM-partially-assembled matrix (FP64).  The local inverse products run on the tensor
    cores with BF16 operand pairs and FP32 accumulation, the coarse solve in FP64."""
    case = latgen.make_case("ring8")
    prob = Problem(case)
    u0 = _u0(prob, 1, 0.0005, 4)
    ul = prob.local(u0)
    rng = np.random.default_rng(21)
    vg = rng.uniform(-1, 1, prob.n_dof)
    vg[prob.fixed] = 0.0
    x_ref, idx, fe, n_r = _oracle_kinv_rom(prob, ul, 1e-2, vg)
    lat = L.Lattice.from_case(case, 2)
    ud = torch.tensor(u0, device="cuda")
    sel = lat.select_principal_cells(ud, 1e-2, 256)
    assert sel["n_r"] == n_r
    lat.lattice_set_timing(True)
    lat.lattice_prepare_solver(ud, lat.lattice_default_opts(eps=1e-2, precond_tangent=0, max_enrich=0))
    s = lat.sizes
    v = lat.feti_from_global(torch.tensor(vg, device="cuda"))
    w = lat.feti_apply(1, v).cpu().numpy()
    _, n_tc = lat.lattice_kernel_time("local_tc")
    lat.lattice_set_timing(False)
    assert n_tc > 0, "the tensor-core product did not run"
    wl = w[: s.n_loc * s.n_cells].reshape(s.n_loc, s.n_cells)
    rmask = fe.r_index >= 0                      # [N_s, n_loc] remaining, non-fixed entries
    got = wl.T[rmask]
    ref = x_ref[idx[rmask]]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-4, err
    lat.close()
