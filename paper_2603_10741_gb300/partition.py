"""Cell-slab partition of a lattice over several ranks and the exchange plan of the FETI-DP
saddle-point operator (host-side index logic).

Cells are independent units for the residual, the snapshots, the greedy's per-cell passes, the
principal tangents and the reduced tangent action; the only couplings of the Krylov loop are the
interface jumps B x and B^T lambda, the primal assembly and the dot products (Section 3.3.1).
With cells split into contiguous slabs of cell layers along the load axis:

* each rank owns the cells of its slab, their rows of every cell-stacked vector and the
  multipliers whose first copy lies in one of its cells;
* B x needs, for an owned multiplier whose second copy lies on another rank, that copy's value
  (halo receive), and B^T lambda sends the multiplier back to the rank of that copy;
* the primal (corner) part is replicated: every rank adds its cells' contributions to the coarse
  right-hand side and one all-reduce (sum) assembles it; the coarse solve is repeated on every
  rank;
* dot products add the owned local rows and owned multipliers of every rank and the primal part
  once (rank 0), then one all-reduce (sum).

The multipliers follow the library's non-redundant reading: a free, non-primal DOF with m copies
(cells, in cell order) gets m - 1 multipliers joining consecutive copies.  This module holds no
arithmetic of the method; it only says which rank holds what and who sends what to whom.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def slab_partition(cell_layer: np.ndarray, n_ranks: int) -> np.ndarray:
    """Rank of every cell: contiguous ranges of cell layers (ascending), balanced by cell count;
    every rank gets at least one layer."""
    cell_layer = np.asarray(cell_layer)
    layers, counts = np.unique(cell_layer, return_counts=True)
    if n_ranks < 1 or n_ranks > layers.size:
        raise ValueError("need 1 <= n_ranks <= number of cell layers")
    total = counts.sum()
    rank_of_layer = np.zeros(layers.size, dtype=np.int64)
    r, cum = 0, 0
    for l in range(layers.size):
        left_layers = layers.size - l
        left_ranks = n_ranks - r
        # move on once this rank has its share, or when every remaining rank needs a layer
        if r < n_ranks - 1 and l > 0 and rank_of_layer[l - 1] == r and \
                (cum >= (r + 1) * total / n_ranks or left_layers < left_ranks):
            r += 1
        rank_of_layer[l] = r
        cum += counts[l]
    lookup = dict(zip(layers.tolist(), rank_of_layer.tolist()))
    return np.array([lookup[v] for v in cell_layer.tolist()], dtype=np.int64)


@dataclasses.dataclass
class ExchangePlan:
    """What rank `rank` holds and exchanges (indices into global FETI-DP numbering)."""
    rank: int
    n_ranks: int
    cells: np.ndarray            # owned cells, ascending
    lam_owned: np.ndarray        # owned multipliers (first copy in an owned cell)
    # B x: for every owned multiplier l, lam = x[first] - x[second]; second copies held by other
    # ranks arrive in recv_x[q] (the multipliers listed in recv_lam[q], in that order)
    recv_lam: dict               # peer rank -> multipliers whose second copy lives on that peer
    send_lam: dict               # peer rank -> multipliers owned by the peer whose second copy is here
    primal_root: bool            # this rank adds the replicated primal part to dot products


@dataclasses.dataclass
class FetiLayout:
    """FETI-DP numbering of the lattice (the library's reading, rebuilt on the host)."""
    n_cells: int
    n_loc: int
    copies_first: np.ndarray     # [n_lambda] local entry (cell, local dof) of the + copy
    copies_second: np.ndarray    # [n_lambda] local entry of the - copy
    cell_of_first: np.ndarray
    cell_of_second: np.ndarray
    primal_dofs: np.ndarray      # free global primal DOFs, ascending (the primal numbering)


def feti_layout(cell_nodes: np.ndarray, dim: int, dof_fixed: np.ndarray, corner_local: np.ndarray) -> FetiLayout:
    """Multipliers and primal DOFs of the lattice: corners primal; every other free DOF shared by
    m > 1 cells gets m - 1 multipliers joining its consecutive copies in cell order."""
    cell_nodes = np.asarray(cell_nodes, dtype=np.int64)
    n_cells, nn = cell_nodes.shape
    n_loc = nn * dim
    is_p = np.zeros(nn, dtype=bool)
    is_p[np.asarray(corner_local, dtype=np.int64)] = True
    gdof = (cell_nodes[:, :, None] * dim + np.arange(dim)).reshape(n_cells, n_loc)
    p_dof = np.repeat(is_p, dim)
    fixed = np.asarray(dof_fixed, dtype=bool)
    rem = (~p_dof)[None, :] & ~fixed[gdof]
    s_idx, k_idx = np.nonzero(rem)                      # cell-major, local dof ascending
    g = gdof[s_idx, k_idx]
    order = np.argsort(g, kind="stable")                # copies of a DOF in cell order
    g_sorted = g[order]
    same = g_sorted[1:] == g_sorted[:-1]
    first = order[:-1][same]
    second = order[1:][same]
    # multipliers numbered in order of the global DOF's first appearance, then copy order
    first_seen = {}
    for pos, dof in enumerate(g.tolist()):
        first_seen.setdefault(dof, pos)
    key = np.array([first_seen[d] for d in g[first].tolist()], dtype=np.int64)
    lam_order = np.lexsort((first, key))
    first, second = first[lam_order], second[lam_order]
    entry = k_idx * n_cells + s_idx                     # cell-stacked position [n_loc][n_cells]
    pg = np.unique(gdof[:, p_dof].ravel())
    pg = pg[~fixed[pg]]
    return FetiLayout(n_cells=n_cells, n_loc=n_loc, copies_first=entry[first], copies_second=entry[second],
                      cell_of_first=s_idx[first], cell_of_second=s_idx[second], primal_dofs=pg)


def exchange_plans(layout: FetiLayout, rank_of_cell: np.ndarray) -> list:
    """One ExchangePlan per rank for the given cell ranks."""
    rank_of_cell = np.asarray(rank_of_cell, dtype=np.int64)
    n_ranks = int(rank_of_cell.max()) + 1
    r1 = rank_of_cell[layout.cell_of_first]
    r2 = rank_of_cell[layout.cell_of_second]
    plans = []
    for r in range(n_ranks):
        owned = np.nonzero(r1 == r)[0]
        recv, send = {}, {}
        for q in range(n_ranks):
            if q == r:
                continue
            rl = owned[r2[owned] == q]
            if rl.size:
                recv[q] = rl
            sl = np.nonzero((r1 == q) & (r2 == r))[0]
            if sl.size:
                send[q] = sl
        plans.append(ExchangePlan(rank=r, n_ranks=n_ranks, cells=np.nonzero(rank_of_cell == r)[0],
                                  lam_owned=owned, recv_lam=recv, send_lam=send, primal_root=(r == 0)))
    return plans
