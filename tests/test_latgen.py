"""Synthetic lattice inputs: sizes, orientation, conformity (CPU)."""
import numpy as np
import pytest

import latgen


def _jac_ok(X, E):
    d = X.shape[1]
    if d == 2:
        a, b, c = X[E[:, 0]], X[E[:, 1]], X[E[:, 3]]
        det = (b - a)[:, 0] * (c - a)[:, 1] - (b - a)[:, 1] * (c - a)[:, 0]
    else:
        a = X[E[:, 0]]
        det = np.linalg.det(np.stack([X[E[:, 1]] - a, X[E[:, 3]] - a, X[E[:, 4]] - a], axis=1))
    return np.all(det > 0)


@pytest.mark.parametrize("n,ne,nn", [(8, 64, 80), (16, 256, 288)])
def test_ring_cell_sizes(n, ne, nn):
    X, E = latgen.ring_cell(n)
    assert E.shape == (ne, 4) and X.shape == (nn, 2)
    assert _jac_ok(X, E)
    corners = np.all((np.abs(X) < 1e-12) | (np.abs(X - 1) < 1e-12), axis=1)
    assert corners.sum() == 4


def test_strut_cell_sizes():
    X, E = latgen.strut_cell(12, 0.15)
    assert E.shape == (344, 8) and X.shape == (880, 3)
    assert _jac_ok(X, E)
    corners = np.all((np.abs(X) < 1e-12) | (np.abs(X - 1) < 1e-12), axis=1)
    assert corners.sum() == 8
    on_face = np.any((np.abs(X) < 1e-12) | (np.abs(X - 1) < 1e-12), axis=1)
    assert on_face.sum() == 572


@pytest.mark.parametrize("name,ndof", [("ring4", 2338), ("ring32", 556034), ("strut10", 1760583)])
def test_lattice_global_dofs(name, ndof):
    c = latgen.make_case(name)
    assert c.lattice.n_nodes * c.lattice.dim == ndof


def test_tiling_conformity():
    c = latgen.make_case("ring4")
    L = c.lattice
    # every global node is used, and coordinates agree between all copies
    Xc = L.cell_origin[:, None, :] + L.X_ref[None]
    assert np.abs(Xc - L.X[L.cell_nodes]).max() < 1e-12
    assert np.unique(L.cell_nodes).size == L.n_nodes


def test_mu_scale_seeded():
    a = latgen.mu_scale(1024, 2)
    assert a.min() >= 0.9 and a.max() <= 1.1
    assert np.array_equal(a, np.random.default_rng(2).uniform(0.9, 1.1, 1024))
