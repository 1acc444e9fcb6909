"""Cell-slab partition and FETI-DP exchange plan over several ranks (CPU, gloo, world size 2).

The sharded saddle-point operator [K~ B^T; B 0] and the sharded dot product (the two pieces of a
Krylov iteration that couple ranks), assembled from the exchange plan with point-to-point halo
messages and sum all-reduces, must equal the single-rank operator and dot of the oracle's
FETI-DP system (Section 3.3.1) on the same vector."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _corner_local(X_ref):
    return np.nonzero(np.all((np.abs(X_ref) < 1e-12) | (np.abs(X_ref - 1) < 1e-12), axis=1))[0]


def _system(name):
    """Oracle FETI-DP pieces of a small lattice at a jittered state: per-cell exact tangents, the
    partially assembled matrix, B, index maps, and the library-reading layout of the partition."""
    import scipy.sparse as sp
    import latgen
    from oracle import cell as OC
    from oracle import newton as ON
    from oracle.assembly import Problem
    from oracle.fetidp import FetiDP
    from paper_2603_10741_gb300 import partition as P
    case = latgen.make_case(name)
    prob = Problem(case)
    u = ON.predictor(prob, 1, None, None)
    u[prob.free] += 0.0005 * latgen.uniform_field(prob.free.size, 3)
    K = OC.tangent(prob.cell, prob.local(u), prob.mu_cells, prob.lam)
    fe = FetiDP(prob)
    idx = fe._index()
    n = fe.n_r + fe.n_p
    ri, ci = idx[:, prob.cell.rows], idx[:, prob.cell.cols]
    keep = (ri >= 0) & (ci >= 0)
    Kt = sp.csr_matrix((K[keep], (ri[keep], ci[keep])), shape=(n, n))
    Bf = sp.hstack([fe.B, sp.csr_matrix((fe.n_lambda, fe.n_p))]).tocsr()
    A = sp.bmat([[Kt, Bf.T], [Bf, None]]).tocsr()
    lat = prob.lat
    lay = P.feti_layout(lat.cell_nodes, prob.d, prob.fixed, _corner_local(lat.X_ref))
    layer = np.round(lat.cell_origin[:, lat.load_axis]).astype(np.int64)
    return prob, K, fe, idx, A, lay, layer


@pytest.mark.parametrize("name", ["ring4", "strut2"])
def test_layout_matches_oracle_multipliers(name):
    prob, K, fe, idx, A, lay, layer = _system(name)
    n_cells = prob.lat.n_cells
    # oracle remaining unknown -> cell-stacked entry
    s_of, k_of = np.nonzero(fe.r_index >= 0)
    entry_of_r = np.empty(fe.n_r, dtype=np.int64)
    entry_of_r[fe.r_index[s_of, k_of]] = k_of * n_cells + s_of
    B = fe.B.tocoo()
    plus = np.zeros(fe.n_lambda, dtype=np.int64)
    minus = np.zeros(fe.n_lambda, dtype=np.int64)
    plus[B.row[B.data > 0]] = B.col[B.data > 0]
    minus[B.row[B.data < 0]] = B.col[B.data < 0]
    assert np.array_equal(entry_of_r[plus], lay.copies_first)
    assert np.array_equal(entry_of_r[minus], lay.copies_second)
    assert np.array_equal(lay.primal_dofs, fe.p_glob)


@pytest.mark.parametrize("n_ranks", [2, 3])
def test_slab_partition_is_contiguous_and_balanced(n_ranks):
    from paper_2603_10741_gb300 import partition as P
    layer = np.repeat(np.arange(6), 7)
    r = P.slab_partition(layer, n_ranks)
    assert np.all(np.diff(r) >= 0) and set(r.tolist()) == set(range(n_ranks))
    counts = np.bincount(r)
    assert counts.max() - counts.min() <= 7


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, name, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2603_10741_gb300 import partition as P
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, K, fe, idx, A, lay, layer = _system(name)
    cell = prob.cell
    n_cells, n_loc = lay.n_cells, lay.n_loc
    n_r, n_p, L = fe.n_r, fe.n_p, fe.n_lambda
    plan = P.exchange_plans(lay, P.slab_partition(layer, world))[rank]
    # the same seeded saddle-point vector on every rank, in the oracle's numbering
    rng = np.random.default_rng(31)
    v = rng.uniform(-1, 1, n_r + n_p + L)
    # its cell-stacked image: local part (remaining rows), replicated primal part, multipliers
    xloc = np.zeros(n_loc * n_cells)
    s_of, k_of = np.nonzero(fe.r_index >= 0)
    xloc[k_of * n_cells + s_of] = v[fe.r_index[s_of, k_of]]
    vP = v[n_r:n_r + n_p]
    lam = v[n_r + n_p:]
    p_of = -np.ones(prob.n_dof, dtype=np.int64)
    p_of[lay.primal_dofs] = np.arange(n_p)

    def exchange(vals_for_peer, peers_recv):
        """Point-to-point halo: send vals_for_peer[q] to q, receive len(peers_recv[q]) from q."""
        reqs, got = [], {}
        for q, arr in vals_for_peer.items():
            reqs.append(dist.isend(torch.tensor(arr, dtype=torch.float64), q))
        for q, cnt in peers_recv.items():
            buf = torch.zeros(cnt, dtype=torch.float64)
            reqs.append(dist.irecv(buf, q))
            got[q] = buf
        for r in reqs:
            r.wait()
        return {q: b.numpy() for q, b in got.items()}

    def sharded_apply(xloc, vP, lam):
        """w = A v on this rank's cells, owned multipliers and the replicated primal part."""
        wloc = np.zeros_like(xloc)
        gP = np.zeros(n_p)
        cd = prob.cell_dofs
        for s in plan.cells:
            Kd = cell.dense(K[s])
            xs = np.zeros(n_loc)
            for k in range(n_loc):
                i = idx[s, k]
                if i < 0:
                    continue
                xs[k] = xloc[k * n_cells + s] if i < n_r else vP[i - n_r]
            ys = Kd @ xs
            for k in range(n_loc):
                i = idx[s, k]
                if i < 0:
                    continue
                if i < n_r:
                    wloc[k * n_cells + s] += ys[k]
                else:
                    gP[p_of[cd[s, k]]] += ys[k]
        # primal assembly: one sum all-reduce (replicated coarse part)
        t = torch.tensor(gP)
        dist.all_reduce(t)
        wP = t.numpy()
        # B^T lambda: first copies are local; second copies of owned multipliers on other ranks
        # are sent there, and multipliers of other ranks with a second copy here are received
        wloc_t = wloc
        for l in plan.lam_owned:
            wloc_t[lay.copies_first[l]] += lam[l]
            if P_rank(l) == rank:
                wloc_t[lay.copies_second[l]] -= lam[l]
        got = exchange({q: lam[ls] for q, ls in plan.recv_lam.items()},
                       {q: len(ls) for q, ls in plan.send_lam.items()})
        for q, vals in got.items():
            for l, val in zip(plan.send_lam[q], vals):
                wloc_t[lay.copies_second[l]] -= val
        # B x: owned multipliers, second copies from their ranks
        got = exchange({q: xloc[lay.copies_second[ls]] for q, ls in plan.send_lam.items()},
                       {q: len(ls) for q, ls in plan.recv_lam.items()})
        second = {}
        for q, vals in got.items():
            second.update(zip(plan.recv_lam[q].tolist(), vals.tolist()))
        wl = {}
        for l in plan.lam_owned:
            sv = xloc[lay.copies_second[l]] if P_rank(l) == rank else second[int(l)]
            wl[int(l)] = xloc[lay.copies_first[l]] - sv
        return wloc_t, wP, wl

    rank_of_cell = P.slab_partition(layer, world)

    def P_rank(l):
        return rank_of_cell[lay.cell_of_second[l]]

    wloc, wP, wl = sharded_apply(xloc, vP, lam)
    # gather the sharded result on every rank and compare with the single-rank operator
    mine = {"loc": {int(e): float(wloc[e]) for s in plan.cells for e in (np.arange(n_loc) * n_cells + s)},
            "lam": wl}
    allp = [None] * world
    dist.all_gather_object(allp, mine)
    ref = A @ v
    ref_loc = np.zeros(n_loc * n_cells)
    ref_loc[k_of * n_cells + s_of] = ref[fe.r_index[s_of, k_of]]
    err = 0.0
    for part in allp:
        for e, val in part["loc"].items():
            err = max(err, abs(val - ref_loc[e]))
        for l, val in part["lam"].items():
            err = max(err, abs(val - ref[n_r + n_p + l]))
    err = max(err, np.abs(wP - ref[n_r:n_r + n_p]).max())
    scale = np.abs(ref).max()
    # sharded dot <v, A v>: owned local rows + owned multipliers, primal part on rank 0, one sum
    d = sum(xloc[k * n_cells + s] * wloc[k * n_cells + s] for s in plan.cells for k in range(n_loc))
    d += sum(lam[l] * wl[int(l)] for l in plan.lam_owned)
    if plan.primal_root:
        d += float(vP @ wP)
    t = torch.tensor([d], dtype=torch.float64)
    dist.all_reduce(t)
    out[rank] = (err / scale, abs(t.item() - v @ ref) / abs(v @ ref), len(plan.cells),
                 sum(len(x) for x in plan.recv_lam.values()))
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["ring4", "strut2"])
def test_sharded_saddle_point_operator_two_gloo_ranks(name):
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, name, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = dict(out)
    for r in range(2):
        op_err, dot_err, n_cells, n_halo = res[r]
        assert op_err < 1e-13, (r, op_err)
        assert dot_err < 1e-12, (r, dot_err)
        assert n_cells > 0
    # the slab boundary cuts interfaces: rank 0 owns multipliers whose second copy is on rank 1
    assert res[0][3] > 0
