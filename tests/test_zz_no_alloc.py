"""The allocation-free greedy entry point agrees with greedy_select (GPU, through the C ABI).

greedy_select_static serves callers that cannot allocate device memory (an arena that owns the
device budget, a host that forbids cudaMalloc, code that cannot create a lattice handle).  This
file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import latgen
from oracle import cell as OC
from oracle.assembly import Problem

pytestmark = pytest.mark.gpu


def _snapshots(seed):
    case = latgen.make_case("ring8")
    prob = Problem(case)
    u = latgen.smooth_state(case.lattice, 0.03, seed).ravel()
    T = OC.snapshots(prob.cell, prob.local(u), prob.mu_cells, prob.lam)      # [nnz, N_s]
    return case, torch.tensor(T.T.copy(), device="cuda")


def test_static_greedy_matches_greedy_select_twice():
    import __graft_entry__ as g
    g.build()
    from paper_2603_10741_gb300 import lattice as L
    for seed in (30, 31):                      # two calls in a row share the static workspace
        case, T = _snapshots(seed)
        lat = L.Lattice.from_case(case)
        ref = lat.greedy_select(T, 1e-3, 64)
        S, alpha = L.greedy_select_static(T, 1e-3, 64)
        torch.cuda.synchronize()
        assert S.cpu().tolist() == ref["S"].cpu().tolist()
        a, b = alpha.cpu().numpy(), ref["alpha"].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1.0)
        lat.close()


def test_static_greedy_rejects_oversized_input():
    import __graft_entry__ as g
    g.build()
    from paper_2603_10741_gb300 import lattice as L
    T = torch.zeros((4096, 1024), dtype=torch.float64, device="cuda")   # 4 Mi entries > 2 Mi
    with pytest.raises(L.LatticeError) as e:
        L.greedy_select_static(T, 1e-3, 8)
    assert e.value.code == 1
