"""GPU parity of the 3D Newton / FETI-DP solve on the edge-strut lattice against the FP64 oracle.

The strut cell (12^3 voxels, struts of half-width 0.15 on the cube edges) puts the cell
interfaces along the struts: under compression the corner-only local remaining blocks of the
full tangent lose definiteness at once (and the global tangent itself is indefinite at the
affine predictor of step 1 and past ~7 % compression on the symmetric branch), so these tests
also pin the preconditioner built from the material part of the principal tangents.  The
operator is the full reduced tangent, so the converged displacements are the oracle's:
1e-10 relative L2 in FP64 (Newton to 1e-12 on both sides), the Newton tolerance in the mixed
modes, with the oracle's own residual evaluated at the GPU solution.
"""
import functools

import numpy as np
import pytest
import torch

import latgen
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
def _oracle_path(name, steps):
    prob = Problem(latgen.make_case(name))
    states, reps = ON.load_path(prob, n_steps=steps, tol=1e-12)
    return prob, states


def test_strut222_load_path_fp64(L):
    """Three load steps (-3 %) on 2 x 2 x 2 strut cells, reduced FP64 path: every converged state
    within 1e-10 (relative L2) of the oracle's."""
    from paper_2603_10741_gb300 import LAT_FP64
    prob, ref = _oracle_path("strut222", 3)
    case = prob.case
    lat = L.Lattice.from_case(case, LAT_FP64)
    opts = lat.lattice_default_opts(newton_rtol=1e-12)
    u1 = u2 = None
    for k in range(1, 4):
        u = lat.lattice_predictor(case.top_displacement(k), u1, u2)
        rep = lat.newton_step(u, opts)
        assert rep.converged, rep.as_dict()
        got = u.cpu().numpy()
        err = np.linalg.norm(got - ref[k - 1]) / np.linalg.norm(ref[k - 1])
        assert err < 1e-10, (k, err)
        u2, u1 = u1, u
    lat.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_strut222_load_path_mixed(L, precision):
    """The same three steps in the mixed modes (FP32 reduced tangent action in the inner Krylov
    solve, FP32 or BF16 preconditioner blocks; FP64 residual, update and outer operator): within
    the Newton tolerance of the oracle, and the oracle's residual at the GPU solution is below
    1e-8 of its residual at the step's predictor."""
    prob, ref = _oracle_path("strut222", 3)
    case = prob.case
    lat = L.Lattice.from_case(case, precision)
    opts = lat.lattice_default_opts()
    u1 = u2 = None
    for k in range(1, 4):
        u = lat.lattice_predictor(case.top_displacement(k), u1, u2)
        rep = lat.newton_step(u, opts)
        assert rep.converged, rep.as_dict()
        assert rep.inner_its_total > 0
        got = u.cpu().numpy()
        err = np.linalg.norm(got - ref[k - 1]) / np.linalg.norm(ref[k - 1])
        assert err < 1e-7, (k, err)
        pred = ON.predictor(prob, k, ref[k - 2] if k > 1 else None, ref[k - 3] if k > 2 else None)
        r = prob.residual(got)
        r0 = prob.residual(pred)
        assert np.linalg.norm(r[prob.free]) <= 1e-8 * np.linalg.norm(r0[prob.free]), k
        u2, u1 = u1, u
    lat.close()


def test_strut10_step1_mixed_full_size(L):
    """Load step 1 of the 10 x 10 x 10 strut lattice (1 000 cells, 1 760 583 DOF) from the affine
    predictor in the mixed FP32 mode: converges, and the oracle's residual at the GPU solution is
    below 1e-8 of the oracle's residual at the predictor."""
    from paper_2603_10741_gb300 import LAT_MIXED_FP32
    case = latgen.make_case("strut10")
    prob = Problem(case)
    lat = L.Lattice.from_case(case, LAT_MIXED_FP32)
    u = lat.lattice_predictor(case.top_displacement(1))
    rep = lat.newton_step(u, lat.lattice_default_opts())
    assert rep.converged, rep.as_dict()
    got = u.cpu().numpy()
    r = prob.residual(got)
    r0 = prob.residual(ON.predictor(prob, 1, None, None))
    assert np.linalg.norm(r[prob.free]) <= 1e-8 * np.linalg.norm(r0[prob.free])
    lat.close()
