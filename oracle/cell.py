"""Per-cell internal force, tangent and snapshots (oracle, FP64).

For a batch of cells with local nodal displacements u [nc, n_nodes, d]:

* deformation gradient, indicial form of Section 3.1.3:
      F_ij = delta_ij + sum_a (d phi_a / d X_j) u_{a,i}
* internal force, Eq. (internalloadvec):  f_a = int sigma grad_x(phi_a) dx,
      grad_x phi = F^{-T} grad_X phi,  dx = J dX
* tangent, Section 3.1.4:  K_ab = int D : (grad_x phi_a (x) grad_x phi_b) dx,
      [K_ab]_ij = sum_kl d_k phi_a D_ijkl d_l phi_b
* snapshot, Eq. (snapshots): data() of the tangent built with the reduced rule.

Local tangents are stored on the shared local sparsity pattern: all node pairs (a, b) that
share an element, sorted by a then b, each pair a d x d block in row-major (i, j) order.
That order is the data() order of the snapshot vectors.
"""
import numpy as np

from . import fe
from .material import cauchy_stress, tangent_tensor_D


class RefCell:
    """Reference-cell discretisation shared by every cell of the lattice."""

    def __init__(self, X_ref, elems):
        self.X = np.asarray(X_ref, dtype=float)
        self.elems = np.asarray(elems, dtype=np.int64)
        self.d = self.X.shape[1]
        self.n_nodes = self.X.shape[0]
        self.n_el = self.elems.shape[0]
        self.nen = self.elems.shape[1]
        self.gradX_full, self.W_full = fe.reference_geometry(self.X, self.elems, 2)
        self.gradX_red, self.W_red = fe.reference_geometry(self.X, self.elems, 1)
        self._build_pattern()

    def quad(self, reduced: bool):
        return (self.gradX_red, self.W_red) if reduced else (self.gradX_full, self.W_full)

    def _build_pattern(self):
        pairs = set()
        for el in self.elems:
            for a in el:
                for b in el:
                    pairs.add((int(a), int(b)))
        blocks = np.array(sorted(pairs), dtype=np.int64)        # [nblk, 2]
        self.blocks = blocks
        d = self.d
        self.nnz = blocks.shape[0] * d * d
        ii, jj = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
        self.rows = (blocks[:, 0, None] * d + ii.ravel()[None, :]).ravel()
        self.cols = (blocks[:, 1, None] * d + jj.ravel()[None, :]).ravel()
        # element entry (e, a, i, b, j) -> pattern position
        key = blocks[:, 0] * self.n_nodes + blocks[:, 1]
        order = np.argsort(key)
        ea = self.elems[:, :, None]
        eb = self.elems[:, None, :]
        bid = order[np.searchsorted(key[order], (ea * self.n_nodes + eb).ravel())]
        bid = bid.reshape(self.n_el, self.nen, self.nen)
        pos = (bid[:, :, None, :, None] * d * d
               + ii[None, None, :, None, :] * d + jj[None, None, :, None, :])
        self.elem_pos = pos                                       # [ne, na, d, nb, d]

    def dense(self, vals):
        """Local pattern values [nnz] -> dense n_loc x n_loc matrix."""
        n = self.n_nodes * self.d
        K = np.zeros((n, n))
        K[self.rows, self.cols] = vals
        return K


def deformation_gradient(cell: RefCell, u, reduced=False):
    gradX, _ = cell.quad(reduced)
    ue = u[:, cell.elems]                                         # [nc, ne, na, d]
    return np.eye(cell.d) + np.einsum("ceai,eqaj->ceqij", ue, gradX)


def min_jacobian(cell: RefCell, u, reduced=False):
    """Smallest det F over all quadrature points of each cell."""
    return np.linalg.det(deformation_gradient(cell, u, reduced)).min(axis=(1, 2))


def internal_force(cell: RefCell, u, mu, lam, reduced=False):
    """f^{int,s}: [nc, n_nodes, d] for local displacements u [nc, n_nodes, d], mu [nc]."""
    gradX, W = cell.quad(reduced)
    F = deformation_gradient(cell, u, reduced)
    J = np.linalg.det(F)
    if np.any(J <= 0):
        raise FloatingPointError("non-positive Jacobian")
    mu_b = np.broadcast_to(np.asarray(mu, dtype=float)[:, None, None], J.shape)
    sig = cauchy_stress(F, mu_b, lam)
    Finv = np.linalg.inv(F)                                       # [.., K, i]
    gradx = np.einsum("ceqki,eqak->ceqai", Finv, gradX)
    dx = J * W[None]
    fe_ = np.einsum("ceqij,ceqaj,ceq->ceai", sig, gradx, dx)
    f = np.zeros((u.shape[0], cell.n_nodes, cell.d))
    for a in range(cell.nen):
        np.add.at(f, (slice(None), cell.elems[:, a]), fe_[:, :, a, :])
    return f


def tangent(cell: RefCell, u, mu, lam, reduced=False, chunk=64):
    """Local tangents K^s on the shared pattern: [nc, nnz]."""
    gradX, W = cell.quad(reduced)
    nc = u.shape[0]
    out = np.zeros((nc, cell.nnz))
    mu = np.asarray(mu, dtype=float)
    for c0 in range(0, nc, chunk):
        uc = u[c0:c0 + chunk]
        F = deformation_gradient(cell, uc, reduced)
        J = np.linalg.det(F)
        if np.any(J <= 0):
            raise FloatingPointError("non-positive Jacobian")
        mu_b = np.broadcast_to(mu[c0:c0 + chunk, None, None], J.shape)
        D = tangent_tensor_D(F, mu_b, lam)
        Finv = np.linalg.inv(F)
        gradx = np.einsum("ceqki,eqak->ceqai", Finv, gradX)
        dx = J * W[None]
        Ke = np.einsum("ceqak,ceqijkl,ceqbl,ceq->ceaibj", gradx, D, gradx, dx)
        blk = out[c0:c0 + chunk]
        np.add.at(blk, (slice(None), cell.elem_pos.reshape(cell.n_el, -1)),
                  Ke.reshape(Ke.shape[0], cell.n_el, -1))
    return out


def snapshots(cell: RefCell, u, mu, lam):
    """Snapshot matrix T = [t^1 ... t^Ns], t^s = data(Kbar^s) with the reduced rule: [nnz, nc]."""
    return tangent(cell, u, mu, lam, reduced=True).T.copy()


def dref_snapshots(cell: RefCell, u, mu, lam):
    """Snapshot matrix of the pulled-back tangent tensor (the Remark after Eq. snapshots):
    t^s = vec({D^ref(xi_q)}) over the one-point rule of every element, [n_el * d^4, nc].

    Eq. (tensorfunctionPulledback) with Psi the map from the element's parameter cube to the
    current configuration, J = dx/dxi = F J0 (J0 = dX/dxi of the reference cell):
        D^ref_ijmn = sum_kl D_ijkl (J^-1)_mk (J^-1)_nl |det J|,
    so that [K_ab]_ij = sum_q w_q sum_mn D^ref_ijmn dphi_a/dxi_m dphi_b/dxi_n (Eq.
    stiffmatPulledback).  Entries ordered (element, i, j, m, n), last fastest."""
    d = cell.d
    xi, _ = fe.gauss_rule(1, d)
    gref = fe.q1_grad_ref(xi)                                     # [1, nen, d]
    Xe = cell.X[cell.elems]                                       # [ne, nen, d]
    J0 = np.einsum("eak,qal->eqkl", Xe, gref)                     # [ne, 1, d, d]
    F = deformation_gradient(cell, u, reduced=True)               # [nc, ne, 1, d, d]
    Jm = np.einsum("ceqkp,eqpl->ceqkl", F, J0)                    # dx_k / dxi_l
    if np.any(np.linalg.det(F) <= 0):
        raise FloatingPointError("non-positive Jacobian")
    Jinv = np.linalg.inv(Jm)                                      # dxi_m / dx_k
    detJ = np.abs(np.linalg.det(Jm))
    mu_b = np.broadcast_to(np.asarray(mu, dtype=float)[:, None, None], detJ.shape)
    D = tangent_tensor_D(F, mu_b, lam)                            # [nc, ne, 1, d, d, d, d]
    Dref = np.einsum("ceqijkl,ceqmk,ceqnl,ceq->ceqijmn", D, Jinv, Jinv, detJ)
    return Dref.reshape(u.shape[0], -1).T.copy()
