"""Reduced local tangents and their action (oracle, FP64).

Eq. (romstiffnessmatrix):  K~^s = sum_r alpha_r^s K^r  with K^r = K^{s_r}(u^{s_r}) the full-rule
tangent of principal cell s_r (Eq. reducedbasis).  Its action on cell-stacked vectors:
    Y[:, s] = sum_r alpha_r^s K^r X[:, s]
"""
import numpy as np
import scipy.sparse as sp


def reduced_tangents(Kp, alpha):
    """K~ values for every cell: Kp [N_r, nnz], alpha [N_r, N_s] -> [N_s, nnz]."""
    return alpha.T @ Kp


def reduced_apply(cell, Kp, alpha, X):
    """Y = reduced tangent action on X [n_loc, N_s] (cell-stacked), dense principal matrices."""
    n_r = Kp.shape[0]
    Y = np.zeros_like(X)
    for r in range(n_r):
        Kr = cell.dense(Kp[r])
        Y += (Kr @ X) * alpha[r][None, :]
    return Y


def assembled(prob, Kcells):
    """Global matrix sum_s A^s K~^s A^{sT} from per-cell pattern values [N_s, nnz]."""
    return sp.csr_matrix((np.asarray(Kcells).ravel(), (prob.K_rows, prob.K_cols)),
                         shape=(prob.n_dof, prob.n_dof))
