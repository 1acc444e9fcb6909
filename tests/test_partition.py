"""Cell-slab partition and FETI-DP exchange plan over several ranks (CPU, gloo, 2 and 3 ranks).

The sharded saddle-point operator [K~ B^T; B 0] and the sharded dot product (the two pieces of a
Krylov iteration that couple ranks), assembled from the exchange plan with point-to-point halo
messages and sum all-reduces, must equal the single-rank operator and dot of the oracle's
FETI-DP system (Section 3.3.1) on the same vector; flexible GMRES iterations built from them
must give the single-rank iterate and residual history."""
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


class _Shard:
    """One rank's share of the FETI-DP saddle-point system of `name` under the slab partition:
    its cells' local rows, the replicated primal part and its owned multipliers.  A sharded
    vector is a full-length array [local n_loc*n_cells | primal n_p | multipliers n_lambda] in
    which only this rank's entries are meaningful (the rest stay zero)."""

    def __init__(self, rank, world, name):
        import torch.distributed as dist
        from paper_2603_10741_gb300 import partition as P
        self.dist = dist
        self.rank = rank
        prob, K, fe, idx, A, lay, layer = _system(name)
        self.prob, self.K, self.fe, self.idx, self.A, self.lay = prob, K, fe, idx, A, lay
        self.cell = prob.cell
        self.n_cells, self.n_loc = lay.n_cells, lay.n_loc
        self.n_r, self.n_p, self.L = fe.n_r, fe.n_p, fe.n_lambda
        self.rank_of_cell = P.slab_partition(layer, world)
        self.plan = P.exchange_plans(lay, self.rank_of_cell)[rank]
        self.p_of = -np.ones(prob.n_dof, dtype=np.int64)
        self.p_of[lay.primal_dofs] = np.arange(self.n_p)
        nl = self.n_loc * self.n_cells
        self.nl = nl
        own = np.zeros(nl, dtype=bool)
        for s in self.plan.cells:
            own[np.arange(self.n_loc) * self.n_cells + s] = True
        self.own_loc = own
        self.own_lam = np.zeros(self.L, dtype=bool)
        self.own_lam[self.plan.lam_owned] = True
        # oracle remaining unknown <-> cell-stacked entry
        self.s_of, self.k_of = np.nonzero(fe.r_index >= 0)
        self.entry_of_r = self.k_of * self.n_cells + self.s_of

    def P_rank(self, l):
        return self.rank_of_cell[self.lay.cell_of_second[l]]

    def to_stacked(self, v):
        """A vector in the oracle's numbering -> its cell-stacked image (every entry)."""
        w = np.zeros(self.nl + self.n_p + self.L)
        w[self.entry_of_r] = v[self.fe.r_index[self.s_of, self.k_of]]
        w[self.nl:self.nl + self.n_p] = v[self.n_r:self.n_r + self.n_p]
        w[self.nl + self.n_p:] = v[self.n_r + self.n_p:]
        return w

    def to_oracle(self, w):
        v = np.zeros(self.n_r + self.n_p + self.L)
        v[self.fe.r_index[self.s_of, self.k_of]] = w[self.entry_of_r]
        v[self.n_r:] = w[self.nl:]
        return v

    def restrict(self, w):
        """Keep this rank's entries of a cell-stacked vector (primal part replicated)."""
        out = w.copy()
        out[:self.nl][~self.own_loc] = 0.0
        out[self.nl + self.n_p:][~self.own_lam] = 0.0
        return out

    def exchange(self, vals_for_peer, peers_recv):
        """Point-to-point halo: send vals_for_peer[q] to q, receive len(peers_recv[q]) from q."""
        import torch
        reqs, got = [], {}
        for q, arr in vals_for_peer.items():
            reqs.append(self.dist.isend(torch.tensor(arr, dtype=torch.float64), q))
        for q, cnt in peers_recv.items():
            buf = torch.zeros(cnt, dtype=torch.float64)
            reqs.append(self.dist.irecv(buf, q))
            got[q] = buf
        for r in reqs:
            r.wait()
        return {q: b.numpy() for q, b in got.items()}

    def apply(self, w):
        """A w on this rank: owned local rows, the replicated primal part (one sum all-reduce),
        owned multipliers; halo messages for B x and B^T lambda."""
        import torch
        lay, plan, n_cells, n_loc = self.lay, self.plan, self.n_cells, self.n_loc
        xloc, vP, lam = w[:self.nl], w[self.nl:self.nl + self.n_p], w[self.nl + self.n_p:]
        wloc = np.zeros(self.nl)
        gP = np.zeros(self.n_p)
        cd = self.prob.cell_dofs
        for s in plan.cells:
            Kd = self.cell.dense(self.K[s])
            xs = np.zeros(n_loc)
            for k in range(n_loc):
                i = self.idx[s, k]
                if i < 0:
                    continue
                xs[k] = xloc[k * n_cells + s] if i < self.n_r else vP[i - self.n_r]
            ys = Kd @ xs
            for k in range(n_loc):
                i = self.idx[s, k]
                if i < 0:
                    continue
                if i < self.n_r:
                    wloc[k * n_cells + s] += ys[k]
                else:
                    gP[self.p_of[cd[s, k]]] += ys[k]
        # primal assembly: one sum all-reduce (replicated coarse part)
        t = torch.tensor(gP)
        self.dist.all_reduce(t)
        wP = t.numpy()
        # B^T lambda: first copies are local; second copies of owned multipliers on other ranks
        # are sent there, and multipliers of other ranks with a second copy here are received
        for l in plan.lam_owned:
            wloc[lay.copies_first[l]] += lam[l]
            if self.P_rank(l) == self.rank:
                wloc[lay.copies_second[l]] -= lam[l]
        got = self.exchange({q: lam[ls] for q, ls in plan.recv_lam.items()},
                            {q: len(ls) for q, ls in plan.send_lam.items()})
        for q, vals in got.items():
            for l, val in zip(plan.send_lam[q], vals):
                wloc[lay.copies_second[l]] -= val
        # B x: owned multipliers, second copies from their ranks
        got = self.exchange({q: xloc[lay.copies_second[ls]] for q, ls in plan.send_lam.items()},
                            {q: len(ls) for q, ls in plan.recv_lam.items()})
        second = {}
        for q, vals in got.items():
            second.update(zip(plan.recv_lam[q].tolist(), vals.tolist()))
        wl = np.zeros(self.L)
        for l in plan.lam_owned:
            sv = xloc[lay.copies_second[l]] if self.P_rank(l) == self.rank else second[int(l)]
            wl[l] = xloc[lay.copies_first[l]] - sv
        out = np.concatenate([wloc, wP, wl])
        return self.restrict(out)

    def dot(self, a, b):
        """Sharded dot product: owned local rows and multipliers, the primal part on rank 0 only,
        one sum all-reduce."""
        import torch
        d = float(a[:self.nl][self.own_loc] @ b[:self.nl][self.own_loc])
        d += float(a[self.nl + self.n_p:][self.own_lam] @ b[self.nl + self.n_p:][self.own_lam])
        if self.plan.primal_root:
            d += float(a[self.nl:self.nl + self.n_p] @ b[self.nl:self.nl + self.n_p])
        t = torch.tensor([d], dtype=torch.float64)
        self.dist.all_reduce(t)
        return t.item()


def _jacobi(sh):
    """A preconditioner local to every rank: the inverse diagonal of the cells' tangents on the
    local rows (a cell-stacked entry belongs to one cell), identity on the primal part and the
    multipliers."""
    d = np.ones(sh.nl + sh.n_p + sh.L)
    for s in range(sh.n_cells):
        Kd = sh.cell.dense(sh.K[s])
        for k in range(sh.n_loc):
            i = sh.idx[s, k]
            if 0 <= i < sh.n_r:
                d[k * sh.n_cells + s] = 1.0 / Kd[k, k]
    return d


def _fgmres(apply, dot, prec, b, m):
    """m iterations of right-preconditioned flexible GMRES from x = 0, classical Gram-Schmidt
    applied twice; returns x_m and the least-squares residual norms."""
    beta = np.sqrt(dot(b, b))
    V, Z = [b / beta], []
    H = np.zeros((m + 1, m))
    res = [beta]
    y = None
    for j in range(m):
        z = prec(V[j])
        Z.append(z)
        w = apply(z)
        for _ in range(2):
            h = np.array([dot(w, V[i]) for i in range(j + 1)])
            for i in range(j + 1):
                w = w - h[i] * V[i]
            H[:j + 1, j] += h
        H[j + 1, j] = np.sqrt(dot(w, w))
        V.append(w / H[j + 1, j])
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        res.append(float(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)))
    x = sum(y[i] * Z[i] for i in range(m))
    return x, res


def _rank_main(rank, world, port, name, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = _Shard(rank, world, name)
    # the same seeded saddle-point vector on every rank, in the oracle's numbering
    rng = np.random.default_rng(31)
    v = rng.uniform(-1, 1, sh.n_r + sh.n_p + sh.L)
    w = sh.apply(sh.restrict(sh.to_stacked(v)))
    ref = sh.A @ v
    ref_w = sh.restrict(sh.to_stacked(ref))
    err = np.abs(w - ref_w).max() / np.abs(ref).max()
    d = sh.dot(sh.restrict(sh.to_stacked(v)), w)
    out[rank] = (err, abs(d - v @ ref) / abs(v @ ref), len(sh.plan.cells),
                 sum(len(x) for x in sh.plan.recv_lam.values()))
    dist.destroy_process_group()


def _fgmres_rank_main(rank, world, port, name, m, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = _Shard(rank, world, name)
    rng = np.random.default_rng(41)
    b = rng.uniform(-1, 1, sh.n_r + sh.n_p + sh.L)
    dj = _jacobi(sh)
    x, res = _fgmres(sh.apply, sh.dot, lambda r: sh.restrict(dj * r), sh.restrict(sh.to_stacked(b)), m)
    # gather this rank's entries into the oracle's numbering on every rank
    parts = [None] * world
    dist.all_gather_object(parts, (sh.own_loc, sh.own_lam, x))
    full = np.zeros_like(x)
    for own_loc, own_lam, xp in parts:
        full[:sh.nl][own_loc] = xp[:sh.nl][own_loc]
        full[sh.nl + sh.n_p:][own_lam] = xp[sh.nl + sh.n_p:][own_lam]
    full[sh.nl:sh.nl + sh.n_p] = x[sh.nl:sh.nl + sh.n_p]
    out[rank] = (sh.to_oracle(full), res)
    dist.destroy_process_group()


def _spawn(target, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (out,)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    return dict(out)


@pytest.mark.parametrize("name", ["ring4", "strut2"])
def test_sharded_saddle_point_operator_two_gloo_ranks(name):
    res = _spawn(_rank_main, 2, name)
    for r in range(2):
        op_err, dot_err, n_cells, n_halo = res[r]
        assert op_err < 1e-13, (r, op_err)
        assert dot_err < 1e-12, (r, dot_err)
        assert n_cells > 0
    # the slab boundary cuts interfaces: rank 0 owns multipliers whose second copy is on rank 1
    assert res[0][3] > 0


@pytest.mark.parametrize("name,world", [("ring4", 2), ("strut2", 2), ("ring4", 3)])
def test_sharded_fgmres_iterations_equal_single_rank(name, world):
    """Eight flexible GMRES iterations on the saddle-point system [K~ B^T; B 0] with a
    preconditioner local to every rank (inverse cell diagonals on the local rows), run sharded over
    gloo ranks (halo messages inside the operator, one all-reduce per dot, replicated primal
    part), give the same iterate and the same residual history as the single-rank iteration on
    the assembled oracle system."""
    m = 8
    res = _spawn(_fgmres_rank_main, world, name, m)
    prob, K, fe, idx, A, lay, layer = _system(name)
    rng = np.random.default_rng(41)
    b = rng.uniform(-1, 1, fe.n_r + fe.n_p + fe.n_lambda)
    # the same preconditioner in the oracle's numbering: inverse diagonal of the owning cell's
    # tangent on every remaining unknown (each belongs to one cell), identity elsewhere
    dj = np.ones_like(b)
    s_of, k_of = np.nonzero(fe.r_index >= 0)
    for s, k in zip(s_of, k_of):
        dj[fe.r_index[s, k]] = 1.0 / prob.cell.dense(K[s])[k, k]
    x_ref, res_ref = _fgmres(lambda v: A @ v, lambda a, c: float(a @ c), lambda r: dj * r, b, m)
    assert res_ref[-1] < 0.9 * res_ref[0]           # the iteration makes progress
    for r in range(world):
        x, hist = res[r]
        assert np.abs(x - x_ref).max() < 1e-10 * np.abs(x_ref).max(), r
        assert np.allclose(hist, res_ref, rtol=1e-10, atol=0), r
