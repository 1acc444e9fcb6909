"""Seeded synthetic inputs for the lattice solver: meshes, lattices, load cases, random fields.

This module holds geometry, topology and random numbers only -- no mechanics, no quadrature,
no solver arithmetic.  Both the FP64 CPU oracle (``oracle/``) and the GPU library
(``paper_2603_10741_gb300``) consume what it produces; neither imports the other.

Cells follow the paper's lattice construction (Section 2.1): one reference cell, repeated by
unit translations (the macro-map is the identity), every cell carrying the same local
discretisation (Section 3.1, identical basis on every cell).  The paper's cells are spline
patches; here the reference cells are bilinear / trilinear (Q1) meshes, which the paper allows
(Section 1: the strategy applies to standard finite elements too).

Reference cells
---------------
* ``ring_cell(n)``  -- 2D unit square with a central circular hole (UC3-like, Section 4),
  meshed as four mapped patches of (n/2) x (n/2) quads: 2n elements around, n/2 radially.
  Node (k, j) = (1 - t_j) C_k + t_j S_k with C_k on the circle (centre (0.5, 0.5), radius
  ``hole_r``; angles uniform, patch p spanning +-45 degrees about the normal of square side p),
  S_k uniformly spaced on the square side and t_j = j / (n/2).
* ``strut_cell(res, radius)`` -- 3D unit cube of res^3 voxels keeping every voxel whose centre
  lies closer than ``radius`` to one of the 12 cube edges (simple-cubic struts on cell edges).

Element node order is the usual Q1 counter-clockwise order (2D) and bottom-then-top face order
(3D); every element has positive Jacobian (checked by ``tests/test_latgen.py``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------------------------
# reference cells
# ----------------------------------------------------------------------------------------------


def ring_cell(n: int, hole_r: float = 0.3):
    """Ring (holed square) reference cell, n x n mapped Q1 quads.  Returns (X [nn,2], E [ne,4])."""
    if n % 2 or n < 2:
        raise ValueError("ring cell resolution must be even")
    h = n // 2                      # elements per square side, and radial layers
    nc = 2 * n                      # nodes around the ring
    X = np.zeros(((h + 1) * nc, 2))
    for k in range(nc):
        side, m = divmod(k, h)
        tau = m / h
        if side == 0:
            S = (tau, 0.0)
        elif side == 1:
            S = (1.0, tau)
        elif side == 2:
            S = (1.0 - tau, 1.0)
        else:
            S = (0.0, 1.0 - tau)
        theta = -0.75 * math.pi + 2.0 * math.pi * k / nc
        C = (0.5 + hole_r * math.cos(theta), 0.5 + hole_r * math.sin(theta))
        for j in range(h + 1):
            t = j / h
            X[j * nc + k] = ((1 - t) * C[0] + t * S[0], (1 - t) * C[1] + t * S[1])
    E = []
    for j in range(h):
        for k in range(nc):
            k1 = (k + 1) % nc
            # local xi runs radially outward (j), eta around the ring (k): positive orientation
            E.append((j * nc + k, (j + 1) * nc + k, (j + 1) * nc + k1, j * nc + k1))
    return X, np.asarray(E, dtype=np.int64)


def strut_cell(res: int = 12, radius: float = 0.15):
    """Edge-strut cube reference cell on a res^3 voxel grid.  Returns (X [nn,3], E [ne,8])."""
    c = (np.arange(res) + 0.5) / res
    keep = []
    for k in range(res):
        for j in range(res):
            for i in range(res):
                p = (c[i], c[j], c[k])
                d = math.inf
                for axis in range(3):
                    o = [q for q in range(3) if q != axis]
                    for a0 in (0.0, 1.0):
                        for a1 in (0.0, 1.0):
                            d = min(d, math.hypot(p[o[0]] - a0, p[o[1]] - a1))
                if d < radius:
                    keep.append((i, j, k))
    corner_ids = {}
    E = []
    offs = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    for (i, j, k) in keep:
        el = []
        for (a, b, cc) in offs:
            key = (i + a, j + b, k + cc)
            if key not in corner_ids:
                corner_ids[key] = len(corner_ids)
            el.append(corner_ids[key])
        E.append(el)
    X = np.zeros((len(corner_ids), 3))
    for key, idx in corner_ids.items():
        X[idx] = np.asarray(key, dtype=float) / res
    return X, np.asarray(E, dtype=np.int64)


def solid_cell(n: int, d: int):
    """Solid unit square / cube meshed with n^d Q1 elements.  Returns (X, E)."""
    if d == 2:
        X = np.array([(i / n, j / n) for j in range(n + 1) for i in range(n + 1)])
        E = [(j * (n + 1) + i, j * (n + 1) + i + 1, (j + 1) * (n + 1) + i + 1, (j + 1) * (n + 1) + i)
             for j in range(n) for i in range(n)]
        return X, np.asarray(E, dtype=np.int64)
    m = n + 1
    X = np.array([(i / n, j / n, k / n) for k in range(m) for j in range(m) for i in range(m)])
    idx = lambda i, j, k: (k * m + j) * m + i
    offs = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    E = [[idx(i + a, j + b, k + c) for (a, b, c) in offs]
         for k in range(n) for j in range(n) for i in range(n)]
    return X, np.asarray(E, dtype=np.int64)


# ----------------------------------------------------------------------------------------------
# lattice tiling
# ----------------------------------------------------------------------------------------------


@dataclasses.dataclass
class Lattice:
    """A lattice of unit-translated copies of one reference cell.

    cell_nodes[s, a] is the global node of local node a in cell s (the Boolean map A^s of
    Eq. (residualvector), stored as an index table).  Cells are numbered lexicographically with x
    fastest; global nodes are numbered in order of first appearance in that cell order.
    """
    dim: int
    dims: tuple                 # cells per direction
    X_ref: np.ndarray           # [n_nodes_cell, d] reference-cell node coordinates
    elems: np.ndarray           # [n_el_cell, 2^d] element -> local node
    cell_nodes: np.ndarray      # [N_s, n_nodes_cell] int64 global node ids
    cell_origin: np.ndarray     # [N_s, d]
    X: np.ndarray               # [n_glob_nodes, d] global node coordinates
    load_axis: int              # axis of the compression (y in 2D, z in 3D)

    @property
    def n_cells(self) -> int:
        return self.cell_nodes.shape[0]

    @property
    def n_nodes(self) -> int:
        return self.X.shape[0]

    @property
    def height(self) -> float:
        return float(self.dims[self.load_axis])

    def bottom_nodes(self) -> np.ndarray:
        return np.nonzero(np.abs(self.X[:, self.load_axis]) < 1e-12)[0]

    def top_nodes(self) -> np.ndarray:
        return np.nonzero(np.abs(self.X[:, self.load_axis] - self.height) < 1e-12)[0]


def tile(X_ref: np.ndarray, elems: np.ndarray, dims) -> Lattice:
    """Tile the reference cell over a dims[0] x dims[1] (x dims[2]) block of unit cells."""
    d = X_ref.shape[1]
    dims = tuple(int(v) for v in dims)
    if len(dims) != d:
        raise ValueError("dims must have one entry per space dimension")
    grids = np.meshgrid(*[np.arange(n) for n in dims[::-1]], indexing="ij")
    origin = np.stack([g.ravel() for g in grids[::-1]], axis=1).astype(float)   # x fastest
    n_s, n_loc = origin.shape[0], X_ref.shape[0]
    Xall = (origin[:, None, :] + X_ref[None, :, :]).reshape(-1, d)
    # cell-boundary node coordinates are exact binary fractions, interior nodes never coincide
    key = np.round(Xall * (1 << 20)).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.ravel()
    order = np.argsort(first, kind="stable")          # renumber by first appearance
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    gid = rank[inv]
    X = np.empty((order.size, d))
    X[gid] = Xall
    return Lattice(dim=d, dims=dims, X_ref=X_ref, elems=elems,
                   cell_nodes=gid.reshape(n_s, n_loc), cell_origin=origin, X=X,
                   load_axis=d - 1)


# ----------------------------------------------------------------------------------------------
# load cases
# ----------------------------------------------------------------------------------------------


@dataclasses.dataclass
class LoadCase:
    """Material, loading and solver settings of one synthetic lattice compression test."""
    name: str
    lattice: Lattice
    mu: float
    lam: float
    mu_scale: np.ndarray        # [N_s] per-cell shear-modulus factor theta_s
    total_strain: float         # compression of the lattice height (0.1 = 10 %)
    n_steps: int
    eps: float                  # reduced-basis tolerance of the greedy selection

    def top_displacement(self, step: int) -> float:
        """Prescribed displacement of the top face along the load axis at load step ``step``."""
        return -(step / self.n_steps) * self.total_strain * self.lattice.height


def mu_scale(n_cells: int, seed) -> np.ndarray:
    """Per-cell shear-modulus factors theta_s ~ U[0.9, 1.1], drawn in cell order (x fastest)."""
    if seed is None:
        return np.ones(n_cells)
    return np.random.default_rng(seed).uniform(0.9, 1.1, n_cells)


def make_case(which: str) -> LoadCase:
    """Named load cases.

    ring4      2D, 4x4 ring cells, 8x8 Q1 each, -10 % in 10 steps, mu=1, lam=4
    ring32     2D, 32x32 ring cells, 16x16 Q1 each, theta ~ U[0.9,1.1] (seed 2), -20 % in 20 steps
    strut10    3D, 10^3 strut cells, -15 % in 15 steps
    strut20    3D, 20^3 strut cells, theta ~ U[0.9,1.1] (seed 4), -20 % in 20 steps
    strut5     3D, 5^3 strut cells, -15 % in 15 steps (small 3D case)
    strut222   3D, 2^3 strut cells of the same 12^3-voxel cell, -15 % in 15 steps (3D parity case)
    ring2 / strut2  tiny lattices for tests (strut2: a coarser 6^3-voxel cell)
    """
    table = {
        "ring4": (ring_cell, (8,), (4, 4), None, 0.10, 10, 3e-4),
        "ring32": (ring_cell, (16,), (32, 32), 2, 0.20, 20, 3e-4),
        "ring8": (ring_cell, (8,), (8, 8), 2, 0.10, 10, 3e-4),
        "ring2": (ring_cell, (4,), (2, 2), 3, 0.05, 2, 3e-4),
        "strut10": (strut_cell, (12, 0.15), (10, 10, 10), None, 0.15, 15, 5e-3),
        "strut20": (strut_cell, (12, 0.15), (20, 20, 20), 4, 0.20, 20, 5e-3),
        "strut5": (strut_cell, (12, 0.15), (5, 5, 5), None, 0.15, 15, 5e-3),
        "strut222": (strut_cell, (12, 0.15), (2, 2, 2), None, 0.15, 15, 5e-3),
        "strut2": (strut_cell, (6, 0.2), (2, 2, 2), 3, 0.05, 2, 5e-3),
    }
    if which not in table:
        raise KeyError(which)
    gen, gargs, dims, seed, strain, steps, eps = table[which]
    Xr, E = gen(*gargs)
    lat = tile(Xr, E, dims)
    return LoadCase(name=which, lattice=lat, mu=1.0, lam=4.0,
                    mu_scale=mu_scale(lat.n_cells, seed), total_strain=strain,
                    n_steps=steps, eps=eps)


# ----------------------------------------------------------------------------------------------
# random vectors
# ----------------------------------------------------------------------------------------------


def uniform_field(shape, seed: int) -> np.ndarray:
    """U[-1, 1] entries (seeded), e.g. the cell-stacked vectors fed to the tangent apply."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, shape)


def dirichlet_coefficients(n_r: int, n_cells: int, seed: int) -> np.ndarray:
    """[n_r, n_cells] reduced-basis coefficients, each column Dirichlet(1,...,1) distributed."""
    return np.random.default_rng(seed).dirichlet(np.ones(n_r), n_cells).T.copy()


def smooth_state(lat: Lattice, amplitude: float, seed: int) -> np.ndarray:
    """A smooth random displacement field [n_nodes, d] (sum of a few low sine modes).

    Used as a synthetic, element-inverting-free deformation state for kernel tests.
    """
    rng = np.random.default_rng(seed)
    d = lat.dim
    ext = np.asarray(lat.dims, dtype=float)
    u = np.zeros((lat.n_nodes, d))
    for _ in range(4):
        k = rng.integers(1, 4, size=d)
        ph = rng.uniform(0, 2 * np.pi, size=d)
        amp = rng.uniform(-1, 1, size=d)
        arg = np.pi * (lat.X / ext) * k + ph
        u += amp * np.prod(np.sin(arg), axis=1, keepdims=True)
    u *= amplitude
    # plus per-node jitter so that no two cells see the same state
    u += 0.1 * amplitude * rng.uniform(-1, 1, size=u.shape)
    return u
