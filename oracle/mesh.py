"""Structured mesh level and the DoF map dof(K, mu) (oracle; test infrastructure only).

Sec. 2: the hierarchy T_0 .. T_L with h_l = gamma h_{l-1}; here uniform boxes
with gamma = 1/2.  Sec. 3 (after Eq. (3.4)) defines the map dof(K, mu) from an
element K and a local number mu in {1..(k+1)(R^+S^)} to the global number, over
all k+1 Gauss-Radau time points.  The local order used here is: time node a
first, then the 3^d Q2 nodes times d components (component fastest), then the
d+1 P1disc coefficients.  The global order is the C-ABI order of stg_inputs.
"""
from __future__ import annotations

import numpy as np

from . import element


class Level:
    def __init__(self, spec, level: int, k: int):
        self.spec = spec
        self.dim = spec.dim
        self.k = k
        self.cells = spec.cells(level)
        self.h = tuple((spec.hi[i] - spec.lo[i]) / self.cells[i] for i in range(self.dim))
        self.r = getattr(spec, "order", 2)                         # velocity order of (Q_r)^d x P_{r-1}disc
        self.nn = tuple(self.r * c + 1 for c in self.cells)      # Q_r nodes per direction
        self.n_nodes = int(np.prod(self.nn))
        self.n_cells = int(np.prod(self.cells))
        self.Shat = len(element.pdisc_exponents(self.r, self.dim)) if self.r != 2 else self.dim + 1
        self.R = self.dim * self.n_nodes
        self.S = self.Shat * self.n_cells
        self.N = (k + 1) * (self.R + self.S)
        self.n_loc_nodes = (self.r + 1) ** self.dim
        self.Rhat = self.dim * self.n_loc_nodes
        self.n_patch = (k + 1) * (self.Rhat + self.Shat)

        # cell multi-indices (n_cells, dim), x fastest
        grids = np.meshgrid(*[np.arange(c) for c in self.cells], indexing="ij")
        self.cell_idx = np.stack([g.ravel(order="F") for g in grids], axis=1)
        # global node number of each local node of each cell (n_cells, 3^d)
        loc = element.local_nodes_r(self.dim, self.r)
        self.cell_nodes = np.zeros((self.n_cells, self.n_loc_nodes), dtype=np.int64)
        for i, l in enumerate(loc):
            g = self.r * self.cell_idx + l
            self.cell_nodes[:, i] = self.node_number(g)
        self.dof = self._dof_map()
        # colour(K) = sum_i (c_i & 1) 2^i: cells of one colour share no Q2 node
        self.colour = np.sum((self.cell_idx & 1) << np.arange(self.dim), axis=1)
        # cells removed by an obstacle (2D): they carry no element matrices; the Q2 nodes that
        # belong to no remaining cell and the P1disc coefficients of removed cells are unknowns
        # without an equation, fixed by identity rows
        self.masked = np.zeros(self.n_cells, dtype=bool)
        box = spec.obstacle_cells(level) if getattr(spec, "obstacle", ()) else ()
        if box:
            cx, cy = self.cell_idx[:, 0], self.cell_idx[:, 1]
            self.masked = (cx >= box[0]) & (cx < box[1]) & (cy >= box[2]) & (cy < box[3])
        fluid_count = np.zeros(self.n_nodes, dtype=np.int64)
        np.add.at(fluid_count, self.cell_nodes[~self.masked].ravel(), 1)
        self.dead_nodes = np.nonzero(fluid_count == 0)[0]

    def node_number(self, g: np.ndarray) -> np.ndarray:
        """Global number of Q2 node multi-indices g (..., dim), x fastest."""
        num = np.zeros(g.shape[:-1], dtype=np.int64)
        stride = 1
        for i in range(self.dim):
            num += g[..., i] * stride
            stride *= self.nn[i]
        return num

    def vel_index(self, a, node, comp):
        return a * (self.R + self.S) + node * self.dim + comp

    def pres_index(self, a, cell, m):
        return a * (self.R + self.S) + self.R + cell * self.Shat + m

    def _dof_map(self) -> np.ndarray:
        """dof[K, mu] for all cells, shape (n_cells, n_patch)."""
        d = self.dim
        out = np.zeros((self.n_cells, self.n_patch), dtype=np.int64)
        cells = np.arange(self.n_cells)
        for a in range(self.k + 1):
            base = a * (self.Rhat + self.Shat)
            for i in range(self.n_loc_nodes):
                for c in range(d):
                    out[:, base + i * d + c] = self.vel_index(a, self.cell_nodes[:, i], c)
            for m in range(self.Shat):
                out[:, base + self.Rhat + m] = self.pres_index(a, cells, m)
        return out

    def boundary_faces(self):
        """List of (direction, side, cell numbers) for every face of the domain boundary."""
        faces = []
        for e in range(self.dim):
            for side in (0, 1):
                target = 0 if side == 0 else self.cells[e] - 1
                faces.append((e, side, np.nonzero(self.cell_idx[:, e] == target)[0]))
        return faces

    def dirichlet_faces(self):
        """(direction, side, cell numbers) of every Dirichlet face of the fluid domain: the
        domain's Dirichlet faces (cells not removed) and the faces of remaining cells whose
        neighbour across that face is removed by the obstacle."""
        out = []
        for e, side, cells in self.boundary_faces():
            if self.is_dirichlet(e, side):
                out.append((e, side, cells[~self.masked[cells]]))
        if self.masked.any():
            stride = [1, self.cells[0], self.cells[0] * (self.cells[1] if self.dim > 1 else 1)]
            for e in range(self.dim):
                for side in (0, 1):
                    step = 1 if side == 1 else -1
                    nb = self.cell_idx[:, e] + step
                    inside = (nb >= 0) & (nb < self.cells[e])
                    nbcell = np.arange(self.n_cells) + step * stride[e]
                    hit = inside & ~self.masked
                    hit[hit] = self.masked[nbcell[hit]]
                    out.append((e, side, np.nonzero(hit)[0]))
        return [f for f in out if len(f[2])]

    def is_dirichlet(self, direction: int, side: int) -> bool:
        return bool(self.spec.dirichlet >> (2 * direction + side) & 1)

    def node_coords(self) -> np.ndarray:
        grids = np.meshgrid(*[self.spec.lo[i] + np.arange(self.nn[i]) * self.h[i] / self.r for i in range(self.dim)],
                            indexing="ij")
        return np.stack([g.ravel(order="F") for g in grids], axis=1)

    def cell_centres(self) -> np.ndarray:
        return np.asarray(self.spec.lo) + (self.cell_idx + 0.5) * np.asarray(self.h)
