"""Global assembly and the Dirichlet split (oracle, FP64).

r(u) = sum_s A^s (f^{int,s}(u^s) - f^{ext,s})      Eq. (residualvector), f^ext = 0 here
K(u) = sum_s A^s K^s(u^s) A^{sT}                     Section 3.1.4
A^s is the Boolean local-to-global map, stored as the table cell_nodes[s, a].
Global vectors are node-major: dof = node * d + component.
"""
import numpy as np
import scipy.sparse as sp

from . import cell as C


class Problem:
    """A lattice + material + boundary conditions, with the oracle's global operators."""

    def __init__(self, case, lateral_rollers=False):
        lat = case.lattice
        self.case = case
        self.lat = lat
        self.cell = C.RefCell(lat.X_ref, lat.elems)
        self.d = lat.dim
        self.n_dof = lat.n_nodes * self.d
        self.mu_cells = case.mu * np.asarray(case.mu_scale, dtype=float)
        self.lam = case.lam
        d = self.d
        self.cell_dofs = (lat.cell_nodes[:, :, None] * d + np.arange(d)).reshape(lat.n_cells, -1)
        # Dirichlet: bottom face clamped, top face: axis component prescribed, others zero
        bot, top = lat.bottom_nodes(), lat.top_nodes()
        fixed = np.zeros(self.n_dof, dtype=bool)
        for n in (bot, top):
            for i in range(d):
                fixed[n * d + i] = True
        if lateral_rollers:
            # extra pins used only to build closed-form test states: zero normal displacement
            # on the lateral faces of the lattice
            for ax in range(d):
                if ax == lat.load_axis:
                    continue
                on = (np.abs(lat.X[:, ax]) < 1e-12) | (np.abs(lat.X[:, ax] - lat.dims[ax]) < 1e-12)
                fixed[np.nonzero(on)[0] * d + ax] = True
        self.fixed = fixed
        self.free = np.nonzero(~fixed)[0]
        self.top_axis_dofs = top * d + lat.load_axis
        self.bot_dofs = np.concatenate([bot * d + i for i in range(d)])
        self._coo = None

    def _pattern_coo(self):
        # global (row, col) of every local tangent entry, built on first use (N_s x nnz each)
        if self._coo is None:
            cd = self.cell_dofs
            self._coo = (cd[:, self.cell.rows].ravel(), cd[:, self.cell.cols].ravel())
        return self._coo

    @property
    def K_rows(self):
        return self._pattern_coo()[0]

    @property
    def K_cols(self):
        return self._pattern_coo()[1]

    def dirichlet_values(self, step):
        """Prescribed global displacement values at fixed DOFs for load step ``step``."""
        g = np.zeros(self.n_dof)
        g[self.top_axis_dofs] = self.case.top_displacement(step)
        return g

    def local(self, u):
        """u^s = A^{sT} u for all cells: [N_s, n_nodes, d]."""
        return u[self.cell_dofs].reshape(self.lat.n_cells, self.cell.n_nodes, self.d)

    def residual(self, u, mu=None):
        mu = self.mu_cells if mu is None else mu
        f = C.internal_force(self.cell, self.local(u), mu, self.lam)
        r = np.zeros(self.n_dof)
        np.add.at(r, self.cell_dofs.ravel(), f.reshape(-1))
        return r

    def tangent(self, u, mu=None):
        mu = self.mu_cells if mu is None else mu
        vals = C.tangent(self.cell, self.local(u), mu, self.lam)
        return sp.csr_matrix((vals.ravel(), (self.K_rows, self.K_cols)),
                             shape=(self.n_dof, self.n_dof))

    def min_jacobian(self, u):
        return C.min_jacobian(self.cell, self.local(u)).min()
