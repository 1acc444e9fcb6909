"""Greedy principal-cell selection (Algorithm 1) and reduced-basis coefficients (oracle, FP64).

Algorithm 1 (Section 3.2.2), on the snapshot matrix T = [t^1 ... t^Ns]:
  Delta_0^s = t^s / ||t^s||_2
  while max_s ||Delta_i^s||_inf > eps:
      s_i  = argmax_s ||Delta_{i-1}^s||_inf        (ties: lowest cell index)
      zeta_i = Delta_{i-1}^{s_i} / ||Delta_{i-1}^{s_i}||_2
      beta_i^s = Delta_{i-1}^s . zeta_i ;  Delta_i^s = Delta_{i-1}^s - beta_i^s zeta_i
Outputs S, Z = {zeta_i}, beta, and the certified decomposition t~^s = ||t^s|| Z beta^s.

RB coefficients (Section 3.2.2): alpha^s = (t_eps^T t_eps)^{-1} t_eps^T t^s with
t_eps = [t^{s_1} ... t^{s_Nr}].  Because span Z = span t_eps, the same projection follows from
the triangular system R alpha^s = ||t^s|| beta^s, R_ir = zeta_i . t^{s_r}; both are computed.
The loop also stops when N_r reaches min(N_s, rows of T) or the caller's max_nr.
"""
import dataclasses

import numpy as np


@dataclasses.dataclass
class GreedyResult:
    S: np.ndarray            # [N_r] principal cell indices, in selection order
    Z: np.ndarray            # [n_nz, N_r] orthonormal basis
    beta: np.ndarray         # [N_r, N_s]
    norms: np.ndarray        # [N_s] ||t^s||_2
    max_res: list            # max_s ||Delta_i^s||_inf before each selection, then the final one


def greedy(T, eps, max_nr=None):
    T = np.asarray(T, dtype=float)
    n_nz, n_s = T.shape
    limit = min(n_s, n_nz) if max_nr is None else min(max_nr, n_s, n_nz)
    norms = np.linalg.norm(T, axis=0)
    Delta = T / norms[None, :]
    S, Z, B, hist = [], [], [], []
    while True:
        inf = np.abs(Delta).max(axis=0)
        m = inf.max()
        hist.append(float(m))
        if not m > eps or len(S) >= limit:
            break
        s_i = int(np.argmax(inf))              # numpy returns the first maximal index
        zeta = Delta[:, s_i] / np.linalg.norm(Delta[:, s_i])
        beta = zeta @ Delta
        Delta = Delta - np.outer(zeta, beta)
        S.append(s_i)
        Z.append(zeta)
        B.append(beta)
    n_r = len(S)
    return GreedyResult(S=np.asarray(S, dtype=np.int64),
                        Z=np.array(Z).T if n_r else np.zeros((n_nz, 0)),
                        beta=np.array(B) if n_r else np.zeros((0, n_s)),
                        norms=norms, max_res=hist)


def alpha_normal_equations(T, S):
    """alpha = (t_eps^T t_eps)^{-1} t_eps^T T  -> [N_r, N_s]."""
    te = T[:, S]
    return np.linalg.solve(te.T @ te, te.T @ T)


def alpha_triangular(T, g: GreedyResult):
    """alpha from R alpha^s = ||t^s|| beta^s with R_ir = zeta_i . t^{s_r} (upper triangular)."""
    R = g.Z.T @ T[:, g.S]
    rhs = g.beta * g.norms[None, :]
    return np.linalg.solve(np.triu(R), rhs)
