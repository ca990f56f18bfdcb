"""Geometric-multigrid V-cycle with the local Vanka smoother (oracle; test infrastructure only).

Sec. 3: GMRES is preconditioned by one V-cycle; on the coarsest partition T_0
a direct solver is applied to J_0 d_0 = b_0; on T_l, l >= 1, J_max pre- and
post-smoothing steps of (S0)-(S3) are applied, the pre-smoothing starting
from d^0 = 0.  Readings: the operators of every level are assembled on that
level (rediscretisation) with w injected at the coarse Q2 nodes; the coarse
correction weight is 1; with Dirichlet data on the whole boundary J has one
constant-pressure null vector per Radau node, and the coarse solve is the
bordered system whose extra rows ask for a zero mean of the cell-constant
pressure coefficients.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble, mesh, transfer, vanka


def inject_w(w_fine: np.ndarray, fine, coarse) -> np.ndarray:
    """Values of w at the coarse Q2 nodes (each coarse node is the fine node 2*g)."""
    d, k = fine.dim, fine.k
    wn = w_fine.reshape(k + 1, fine.n_nodes, d)
    grids = np.meshgrid(*[np.arange(n) for n in coarse.nn], indexing="ij")
    g = np.stack([gg.ravel(order="F") for gg in grids], axis=1)
    return wn[:, fine.node_number(2 * g), :].reshape(k + 1, -1)


def pressure_mean_vectors(lev) -> np.ndarray:
    """(k+1, N) rows: area-weighted sum of the cell-constant pressure coefficient per Radau node."""
    c = np.zeros((lev.k + 1, lev.N))
    area = np.prod(lev.h)
    for a in range(lev.k + 1):
        c[a, lev.pres_index(a, np.arange(lev.n_cells), 0)] = area
    return c


def normalise_pressure(lev, x: np.ndarray) -> np.ndarray:
    """Remove the mean of the cell-constant pressure coefficients per Radau node."""
    x = np.array(x, dtype=float, copy=True)
    for a in range(lev.k + 1):
        idx = lev.pres_index(a, np.arange(lev.n_cells), 0)
        x[idx] -= x[idx].mean()
    return x


class Hierarchy:
    """All levels of one slab problem: J_l, local inverses, prolongations, coarse solver."""

    def __init__(self, spec, k: int, nu: float, tau: float, w_fine: np.ndarray, newton: bool = False,
                 omega: float = 0.7, nu1: int = 4, nu2: int = 4, smoother: str = "averaged",
                 gamma1=assemble.GAMMA1, gamma2=assemble.GAMMA2):
        self.spec, self.k, self.nu, self.tau = spec, k, nu, tau
        self.omega, self.nu1, self.nu2, self.smoother = omega, nu1, nu2, smoother
        self.levels = [mesh.Level(spec, l, k) for l in range(spec.n_levels)]
        self.w = [None] * spec.n_levels
        self.w[-1] = np.asarray(w_fine, float).reshape(k + 1, -1)
        for l in range(spec.n_levels - 1, 0, -1):
            self.w[l - 1] = inject_w(self.w[l], self.levels[l], self.levels[l - 1])
        self.J = [assemble.jacobian(lev, self.w[l], nu, tau, newton, gamma1, gamma2)
                  for l, lev in enumerate(self.levels)]
        self.jinv = [None] + [vanka.local_inverses(self.J[l], self.levels[l]) for l in range(1, spec.n_levels)]
        self.P = [None] + [transfer.prolongation(self.levels[l - 1], self.levels[l])
                           for l in range(1, spec.n_levels)]
        self.singular = spec.pure_dirichlet()
        j0 = self.J[0]
        if self.singular:
            c = pressure_mean_vectors(self.levels[0])
            z = sp.csr_matrix((c.shape[0], c.shape[0]))
            j0 = sp.bmat([[j0, sp.csr_matrix(c.T)], [sp.csr_matrix(c), z]], format="csc")
        self._coarse_n = j0.shape[0]
        if j0.shape[0] <= 4000:
            self._coarse_lu = sla.lu_factor(j0.toarray())
            self._coarse_sparse = None
        else:
            self._coarse_lu = None
            self._coarse_sparse = spla.splu(sp.csc_matrix(j0))

    @property
    def fine(self):
        return self.levels[-1]

    def coarse_solve(self, b0: np.ndarray) -> np.ndarray:
        n = self.levels[0].N
        rhs = np.zeros(self._coarse_n)
        rhs[:n] = b0
        if self._coarse_lu is not None:
            sol = sla.lu_solve(self._coarse_lu, rhs)
        else:
            sol = self._coarse_sparse.solve(rhs)
        return sol[:n]

    def smooth(self, level: int, b: np.ndarray, d: np.ndarray, sweeps: int) -> np.ndarray:
        lev = self.levels[level]
        if self.smoother == "averaged":
            return vanka.sweep_averaged(self.J[level], lev, self.jinv[level], b, d, self.omega, sweeps)
        return vanka.sweep_coloured(self.J[level], lev, self.jinv[level], b, d, self.omega, sweeps)

    def vcycle(self, b: np.ndarray, level: int | None = None) -> np.ndarray:
        """One V-cycle d = V(l, b) with d^0 = 0."""
        level = len(self.levels) - 1 if level is None else level
        if level == 0:
            return self.coarse_solve(b)
        d = self.smooth(level, b, np.zeros_like(b), self.nu1)          # pre-smoothing from d^0 = 0
        r = b - self.J[level] @ d
        dc = self.vcycle(self.P[level].T @ r, level - 1)                 # restriction R = P^T
        d = d + self.P[level] @ dc                                       # prolongation, weight 1
        return self.smooth(level, b, d, self.nu2)                        # post-smoothing

    def apply(self, x: np.ndarray) -> np.ndarray:
        return self.J[-1] @ x
