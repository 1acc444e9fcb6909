"""Pins of the oracle's Algorithm 1, RB coefficients and reduced apply -- CPU."""
import numpy as np
import pytest

import latgen
from oracle import cell as C
from oracle import greedy as G
from oracle import rom


def _lowrank(n_nz=40, n_s=15, rank=6, noise=1e-3, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n_nz, rank)) @ rng.normal(size=(rank, n_s)) + noise * rng.normal(size=(n_nz, n_s))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_greedy_matches_brute_force_projection(seed):
    T = _lowrank(seed=seed)
    g = G.greedy(T, 1e-2)
    That = T / np.linalg.norm(T, axis=0)
    for i, s_i in enumerate(g.S):
        # residual of every normalised snapshot after projecting on the previous selections,
        # computed from scratch with a Householder QR instead of the running MGS update
        if i == 0:
            res = That
        else:
            Q, _ = np.linalg.qr(That[:, g.S[:i]])
            res = That - Q @ (Q.T @ That)
        inf = np.abs(res).max(axis=0)
        assert s_i == int(np.argmax(inf))
        assert abs(inf.max() - g.max_res[i]) < 1e-12
    assert g.max_res[-1] <= 1e-2 < g.max_res[-2]


def test_greedy_invariants():
    T = _lowrank(seed=3)
    eps = 5e-3
    g = G.greedy(T, eps)
    n_r = g.S.size
    assert np.abs(g.Z.T @ g.Z - np.eye(n_r)).max() < 1e-12
    # certified decomposition: ||t^s - ||t^s|| Z beta^s||_inf <= eps ||t^s||_2
    approx = g.Z @ g.beta * g.norms[None, :]
    assert np.all(np.abs(T - approx).max(axis=0) <= eps * g.norms * (1 + 1e-12))
    a1 = G.alpha_normal_equations(T, g.S)
    a2 = G.alpha_triangular(T, g)
    assert np.abs(a1 - a2).max() < 1e-9 * np.abs(a1).max()
    assert np.abs(a1[:, g.S] - np.eye(n_r)).max() < 1e-10
    # alpha reproduces the projection: t_eps alpha^s = t~^s
    assert np.abs(T[:, g.S] @ a2 - approx).max() < 1e-10 * np.abs(T).max()


def test_identical_cells_give_one_principal():
    rng = np.random.default_rng(4)
    t = rng.normal(size=50)
    scale = rng.uniform(0.5, 2.0, 9)
    T = np.outer(t, scale)
    g = G.greedy(T, 1e-10)
    assert g.S.size == 1 and g.S[0] == int(np.argmax(np.abs(T / np.linalg.norm(T, axis=0)).max(axis=0)))
    a = G.alpha_triangular(T, g)
    assert np.abs(a[0] - scale / scale[g.S[0]]).max() < 1e-12


def test_tie_break_lowest_index_and_limit():
    T = np.eye(4)
    g = G.greedy(T, 0.1)
    assert list(g.S) == [0, 1, 2, 3]
    g2 = G.greedy(T, 0.1, max_nr=2)
    assert list(g2.S) == [0, 1]


def test_reduced_apply_special_cases():
    X, E = latgen.ring_cell(4)
    cell = C.RefCell(X, E)
    rng = np.random.default_rng(5)
    n_s = 6
    u = 0.01 * rng.uniform(-1, 1, (n_s, cell.n_nodes, 2))
    K = C.tangent(cell, u, np.ones(n_s), 4.0)
    Xv = rng.uniform(-1, 1, (cell.n_nodes * 2, n_s))
    # every cell principal, alpha = I: the per-cell full apply
    Y = rom.reduced_apply(cell, K, np.eye(n_s), Xv)
    for s in range(n_s):
        assert np.abs(Y[:, s] - cell.dense(K[s]) @ Xv[:, s]).max() < 1e-12
    # one principal: a scalar multiple of its apply
    a = rng.uniform(0.5, 1.5, (1, n_s))
    Y1 = rom.reduced_apply(cell, K[2:3], a, Xv)
    assert np.abs(Y1 - a * (cell.dense(K[2]) @ Xv)).max() < 1e-12
    # explicit reduced tangents agree with the action
    al = rng.uniform(-1, 1, (3, n_s))
    Kt = rom.reduced_tangents(K[:3], al)
    Y3 = rom.reduced_apply(cell, K[:3], al, Xv)
    for s in range(n_s):
        assert np.abs(Y3[:, s] - cell.dense(Kt[s]) @ Xv[:, s]).max() < 1e-12
