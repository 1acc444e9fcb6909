"""Q1 reference-element shape functions and Gauss-Legendre quadrature (oracle, FP64).

The paper integrates element by element with (p+1)^d Gauss-Legendre points (Section 3.1.5,
Eq. fullquadraturerule); for the Q1 (p = 1) cells used here that is 2^d points.  The snapshot
rule of Eq. (snapshots) uses fewer points per direction: one point (the element centre).
All cells are unit translates of one reference cell, so the reference gradients and weights
computed here are shared by every cell (the pull-back of Eq. stiffmatPulledback with an
identity macro-map).
"""
import itertools

import numpy as np


def gauss_rule(n_per_dir: int, d: int):
    """Tensor Gauss-Legendre rule on [-1,1]^d: (points [nq,d], weights [nq])."""
    x, w = np.polynomial.legendre.leggauss(n_per_dir)
    pts, wts = [], []
    for idx in itertools.product(range(n_per_dir), repeat=d):
        pts.append([x[i] for i in idx[::-1]])      # first coordinate fastest
        wts.append(np.prod([w[i] for i in idx]))
    return np.asarray(pts), np.asarray(wts)


def q1_nodes(d: int) -> np.ndarray:
    """Local node positions of the Q1 element in [-1,1]^d, counter-clockwise / bottom-then-top."""
    if d == 2:
        return np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=float)
    base = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=float)
    return np.vstack([np.hstack([base, -np.ones((4, 1))]), np.hstack([base, np.ones((4, 1))])])


def q1_grad_ref(xi: np.ndarray) -> np.ndarray:
    """Gradients d phi_a / d xi at points xi [nq,d] -> [nq, 2^d, d] for phi_a = prod(1+xi_a xi)/2^d."""
    nq, d = xi.shape
    na = q1_nodes(d)
    g = np.zeros((nq, na.shape[0], d))
    for a in range(na.shape[0]):
        for k in range(d):
            val = np.full(nq, na[a, k] / 2 ** d)
            for m in range(d):
                if m != k:
                    val = val * (1 + na[a, m] * xi[:, m])
            g[:, a, k] = val
    return g


def q1_shape(xi: np.ndarray) -> np.ndarray:
    """Shape function values [nq, 2^d] at points xi [nq,d]."""
    na = q1_nodes(xi.shape[1])
    return np.prod(1 + na[None, :, :] * xi[:, None, :], axis=2) / 2 ** xi.shape[1]


def reference_geometry(X_ref: np.ndarray, elems: np.ndarray, n_per_dir: int):
    """Per element and quadrature point: gradX [ne,nq,2^d,d] = d phi_a / dX and weight W [ne,nq].

    W = w_q |det J0| with J0 = dX/dxi the element map of the reference cell.
    """
    d = X_ref.shape[1]
    xi, w = gauss_rule(n_per_dir, d)
    gref = q1_grad_ref(xi)                                   # [nq, na, d]
    Xe = X_ref[elems]                                        # [ne, na, d]
    J0 = np.einsum("eak,qal->eqkl", Xe, gref)                # dX_k / dxi_l
    detJ0 = np.linalg.det(J0)
    if np.any(detJ0 <= 0):
        raise ValueError("reference element with non-positive Jacobian")
    J0inv = np.linalg.inv(J0)                                # dxi_l / dX_k  -> [e,q,l,k]
    gradX = np.einsum("qal,eqlk->eqak", gref, J0inv)
    return gradX, w[None, :] * detJ0
