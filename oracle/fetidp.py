"""FETI-DP saddle-point system of the tangent problem, solved directly (oracle, FP64).

Section 3.3.1: each cell is a subdomain; local DOFs split into primal P (cell corners, assembled
globally) and remaining R (interior and dual interface DOFs, kept per cell).  Continuity of the
dual DOFs is imposed by Lagrange multipliers through the signed Boolean jump matrix B:

    [ K~  B^T ] [du    ]   [ -r ]
    [ B   0   ] [lambda] = [  0 ]

K~ is the partially assembled tangent built from per-cell matrices (exact K^s or the reduced
K~^s of Eq. romstiffnessmatrix).  The local residual parts stay unassembled on R and are
assembled on P; any such split sums to the global residual, so du equals the solution of the
assembled system.  Multipliers: a dual DOF with m copies gets m - 1 of them, joining consecutive
copies in cell order (non-redundant, so the saddle point is non-singular and a direct solve
applies); none on Dirichlet DOFs.  This module exists to check the statement above, not to be
fast.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def corner_nodes(X_ref):
    on = np.all((np.abs(X_ref) < 1e-12) | (np.abs(X_ref - 1) < 1e-12), axis=1)
    return np.nonzero(on)[0]


class FetiDP:
    def __init__(self, prob):
        self.prob = prob
        lat, d = prob.lat, prob.d
        n_s, nn = lat.cell_nodes.shape
        corners = corner_nodes(lat.X_ref)
        is_p = np.zeros(nn, dtype=bool)
        is_p[corners] = True
        self.is_p_dof = np.repeat(is_p, d)
        cd = prob.cell_dofs                                    # [N_s, n_loc]
        fixed = prob.fixed
        # remaining DOFs: one unknown per (cell, local R dof) that is not fixed
        r_mask = (~self.is_p_dof)[None, :] & ~fixed[cd]
        self.r_index = -np.ones(cd.shape, dtype=np.int64)
        self.r_index[r_mask] = np.arange(r_mask.sum())
        self.n_r = int(r_mask.sum())
        # primal DOFs: global corner DOFs that are not fixed
        p_glob = np.unique(cd[:, self.is_p_dof].ravel())
        p_glob = p_glob[~fixed[p_glob]]
        self.p_glob = p_glob
        self.p_index = -np.ones(prob.n_dof, dtype=np.int64)
        self.p_index[p_glob] = np.arange(p_glob.size)
        self.n_p = p_glob.size
        # multipliers: consecutive copies of each free, non-primal global DOF shared by >1 cell
        owners = {}
        for s in range(n_s):
            for a in np.nonzero(r_mask[s])[0]:
                owners.setdefault(int(cd[s, a]), []).append(int(self.r_index[s, a]))
        rows, cols, vals = [], [], []
        L = 0
        for g, copies in owners.items():
            for i in range(len(copies) - 1):
                rows += [L, L]
                cols += [copies[i], copies[i + 1]]
                vals += [1.0, -1.0]
                L += 1
        self.n_lambda = L
        self.B = sp.csr_matrix((vals, (rows, cols)), shape=(L, self.n_r))

    def _index(self):
        """Partially assembled unknown index of every (cell, local dof), -1 if fixed."""
        prob = self.prob
        idx = self.r_index.copy()
        cd = prob.cell_dofs
        pmask = self.is_p_dof[None, :] & (self.p_index[cd] >= 0)
        idx[pmask] = self.n_r + self.p_index[cd][pmask]
        return idx

    def solve(self, Kcells, f_cells):
        """Solve the saddle point for per-cell matrices [N_s, nnz] and local residuals [N_s, n_loc].

        Returns (du global [n_dof], lambda [L]); du is zero on fixed DOFs.
        """
        prob, cell = self.prob, self.prob.cell
        idx = self._index()
        n = self.n_r + self.n_p
        ri = idx[:, cell.rows]
        ci = idx[:, cell.cols]
        keep = (ri >= 0) & (ci >= 0)
        Kt = sp.csr_matrix((np.asarray(Kcells)[keep], (ri[keep], ci[keep])), shape=(n, n))
        rhs = np.zeros(n)
        ok = idx >= 0
        np.add.at(rhs, idx[ok], -np.asarray(f_cells)[ok])
        Bfull = sp.hstack([self.B, sp.csr_matrix((self.n_lambda, self.n_p))])
        A = sp.bmat([[Kt, Bfull.T], [Bfull, None]], format="csc")
        sol = spla.splu(A).solve(np.concatenate([rhs, np.zeros(self.n_lambda)]))
        du = np.zeros(prob.n_dof)
        cd = prob.cell_dofs
        du[cd[ok]] = sol[idx[ok]]
        return du, sol[n:]
