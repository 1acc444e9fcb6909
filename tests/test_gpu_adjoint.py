"""GPU adjoint gradient of the end compliance w.r.t. per-cell shear-modulus factors (the
differentiation growth pattern; not in the paper), against the FP64 oracle's direct adjoint and
central finite differences, with load-step checkpointing and the torch autograd wrapper.

J(theta) = u_D . f_D(u(theta)) is evaluated at the end state of the load path; on a fixed branch
of this hyperelastic problem the end state depends only on the final load, so a perturbed J is
the end state re-converged from the unperturbed one (Newton to 1e-13 of the perturbation's
residual)."""
import functools
import os

import numpy as np
import pytest
import torch

import latgen
from oracle import adjoint as OA
from oracle import newton as ON
from oracle.assembly import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    from paper_2603_10741_gb300 import lattice
    return lattice


@functools.lru_cache(maxsize=None)
def _oracle_end(name, steps):
    prob = Problem(latgen.make_case(name))
    states, _ = ON.load_path(prob, n_steps=steps, tol=1e-13)
    return prob, states


def _fd_gradient(lat, case, u_end, theta, cells, h, opts, log=None):
    """Central differences of J over theta_s for the listed cells, re-converging the end state."""
    out = []
    for s in cells:
        if log is not None:
            log("fd cell", int(s))
        vals = []
        for sgn in (1.0, -1.0):
            th = theta.copy()
            th[s] += sgn * h
            lat.lattice_set_mu_scale(th)
            u = u_end.clone()
            rep = lat.newton_step(u, opts)
            assert rep.converged, rep.as_dict()
            r = lat.assemble_residual_tangent(u)["r"].cpu().numpy()
            ud = u.cpu().numpy()
            fixed = lat_fixed(case)
            vals.append(float(ud[fixed] @ r[fixed]))
        out.append((vals[0] - vals[1]) / (2 * h))
    lat.lattice_set_mu_scale(theta)
    return np.asarray(out)


def lat_fixed(case):
    lat = case.lattice
    d = lat.dim
    fixed = np.zeros(lat.n_nodes * d, dtype=bool)
    for n in (lat.bottom_nodes(), lat.top_nodes()):
        for i in range(d):
            fixed[n * d + i] = True
    return fixed


def test_adjoint_strut222_matches_oracle_and_fd(L):
    """2 x 2 x 2 edge-strut cells after three load steps (-3 %), FP64: the GPU gradient w.r.t.
    the 8 per-cell factors equals the oracle's direct adjoint (1e-9 of its largest entry) and
    central differences (h = 1e-5) of the GPU's own J on 4 seeded cells (1e-6)."""
    from paper_2603_10741_gb300 import LAT_FP64
    prob, states = _oracle_end("strut222", 3)
    case = prob.case
    u_ref = states[-1]
    g_ref = OA.gradient(prob, u_ref)
    lat = L.Lattice.from_case(case, LAT_FP64)
    opts = lat.lattice_default_opts(newton_rtol=1e-13)
    from paper_2603_10741_gb300 import solve_load_path
    u, _ = solve_load_path(lat, case, opts, steps=3)
    g, J, rep = lat.adjoint_gradient(u, opts)
    assert rep.converged
    g = g.cpu().numpy()
    assert abs(J - ON.compliance(prob, u_ref)) < 1e-10 * abs(J)
    assert np.abs(g - g_ref).max() < 1e-9 * np.abs(g_ref).max()
    cells = np.sort(np.random.default_rng(5).choice(case.lattice.n_cells, 4, replace=False))
    fd = _fd_gradient(lat, case, u, np.asarray(case.mu_scale, dtype=float), cells, 1e-5, opts)
    assert np.abs(fd - g[cells]).max() < 1e-6 * np.abs(g).max(), (fd, g[cells])
    lat.close()


def test_checkpoint_resume_gives_identical_gradient(L, tmp_path):
    """ring4, FP64: the load path saved step by step; resuming after step 2 from its checkpoint
    reaches step 3 with the same displacement and the same gradient, bit for bit."""
    from paper_2603_10741_gb300 import LAT_FP64, solve_load_path
    case = latgen.make_case("ring4")
    lat = L.Lattice.from_case(case, LAT_FP64)
    opts = lat.lattice_default_opts(newton_rtol=1e-12)
    u_full, _ = solve_load_path(lat, case, opts, steps=3, checkpoint_dir=str(tmp_path))
    g_full, J_full, _ = lat.adjoint_gradient(u_full, opts)
    step, load, u2, u1 = lat.lattice_checkpoint_load(tmp_path / "step_0002.ckpt")
    assert step == 2 and load == case.top_displacement(2)
    lat2 = L.Lattice.from_case(case, LAT_FP64)
    u_res, _ = solve_load_path(lat2, case, opts, steps=3, start=(2, u2, u1))
    g_res, J_res, _ = lat2.adjoint_gradient(u_res, opts)
    assert torch.equal(u_full, u_res)
    assert torch.equal(g_full, g_res) and J_full == J_res
    lat.close()
    lat2.close()


def test_compliance_autograd_function(L):
    """solver.Compliance: torch.autograd.grad of J(theta) through the load path on the 2 x 2 ring
    lattice equals the oracle's adjoint gradient at its own end state."""
    from paper_2603_10741_gb300 import LAT_FP64
    from paper_2603_10741_gb300.solver import Compliance
    prob, states = _oracle_end("ring2", 2)
    case = prob.case
    g_ref = OA.gradient(prob, states[-1])
    lat = L.Lattice.from_case(case, LAT_FP64)
    opts = lat.lattice_default_opts(newton_rtol=1e-13, eps=1e-4)
    theta = torch.tensor(np.asarray(case.mu_scale, dtype=float), dtype=torch.float64, requires_grad=True)
    J = Compliance.apply(theta, lat, case, opts)
    (grad,) = torch.autograd.grad(J, theta)
    assert abs(J.item() - ON.compliance(prob, states[-1])) < 1e-10 * abs(J.item())
    assert np.abs(grad.numpy() - g_ref).max() < 1e-9 * np.abs(g_ref).max()
    lat.close()


@pytest.mark.skipif(os.environ.get("LATTICE_CFG5") != "1",
                    reason="full-size adjoint run (more than 30 minutes of GPU time): set LATTICE_CFG5=1")
def test_cfg5_strut10_adjoint_full_size(L, tmp_path):
    """The adjoint configuration at full size: 10 x 10 x 10 strut cells at -15 % in 15 steps, the
    gradient w.r.t. the 1 000 per-cell factors, with a checkpoint after every load step; central
    differences (h = 1e-6) on the 20 cells rng(5).choice(1000, 20); the gradient after resuming
    from the step-14 checkpoint is identical.  The adjoint is FP64 (defect correction with the
    exact FP64 tangent action, the correction solved by FGMRES on the FP64 reduced operator); its
    preconditioner runs with BF16 blocks, as does the load path's (an FP64 preconditioner would
    make each interface iteration ~20x slower on these 2616-DOF local blocks)."""
    import time
    from paper_2603_10741_gb300 import LAT_MIXED_BF16, solve_load_path
    t0 = time.time()

    def say(*a):
        print("[cfg5 %.0f s]" % (time.time() - t0), *a, flush=True)

    case = latgen.make_case("strut10")
    lat = L.Lattice.from_case(case, LAT_MIXED_BF16)
    opts = lat.lattice_default_opts()               # Newton to 1e-8 relative, as in the configuration
    u, reps = solve_load_path(lat, case, opts, checkpoint_dir=str(tmp_path),
                              log=lambda k, r: say("step", k, "its", r.iterations, "N_r", r.n_r_last,
                                                   "eps", r.eps_last, "refinements", r.eps_refinements))
    # the perturbed end states: 1e-8 of a residual that is itself O(h) after the perturbation
    opts_fd = lat.lattice_default_opts()
    g, J, rep = lat.adjoint_gradient(u, opts_fd)
    say("adjoint", rep.as_dict())
    assert rep.converged
    g = g.cpu().numpy()
    cells = np.random.default_rng(5).choice(1000, 20, replace=False)
    fd = _fd_gradient(lat, case, u, np.asarray(case.mu_scale, dtype=float), cells, 1e-6, opts_fd, log=say)
    say("fd", np.abs(fd - g[cells]).max() / np.abs(g).max())
    assert np.abs(fd - g[cells]).max() < 1e-5 * np.abs(g).max(), (fd, g[cells])
    step, _, u14, u13 = lat.lattice_checkpoint_load(tmp_path / "step_0014.ckpt")
    lat2 = L.Lattice.from_case(case, LAT_MIXED_BF16)
    u_res, _ = solve_load_path(lat2, case, opts, start=(step, u14, u13))
    assert torch.equal(u, u_res)
    g2, _, _ = lat2.adjoint_gradient(u_res, opts_fd)
    assert np.array_equal(g, g2.cpu().numpy())
    say("resumed from step 14: identical displacement and gradient")
    lat.close()
    lat2.close()
