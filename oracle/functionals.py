"""Drag and lift on an obstacle (oracle; test infrastructure only).

Sec. 4 reports drag and lift coefficients of the flow around an obstacle, computed by
approximating the surface integrals that define the forces (the benchmark's definitions).
Reading: the force of the fluid on the obstacle S at Radau node a is

    F = - int_S (nu grad v_h - p_h I) n dS,

with T = nu grad v - p I the stress of the do-nothing form (Sec. 1) and n the unit normal of
the fluid domain on S (pointing into the obstacle); drag F_D = F_x, lift F_L = F_y; the
coefficients are c = 2 F / (U_mean^2 D) with U_mean the mean inflow speed and D the obstacle's
height (rho = 1).  The integrals use the 3-point Gauss rule on each face of the fluid cells
that border the obstacle, with v_h and p_h from those cells.
"""
from __future__ import annotations

import numpy as np

from . import element


def obstacle_forces(lev, X: np.ndarray, nu: float) -> np.ndarray:
    """(k+1, 2) forces (F_x, F_y) on the obstacle at every Radau node of slab vector X."""
    d, k = lev.dim, lev.k
    assert d == 2
    h = np.asarray(lev.h)
    out = np.zeros((k + 1, d))
    if not lev.masked.any():
        return out
    for e, side, cells in lev.dirichlet_faces():
        # faces towards the obstacle: the neighbour cell lies inside the domain and is removed
        nb = lev.cell_idx[cells, e] + (1 if side else -1)
        inside = (nb >= 0) & (nb < lev.cells[e])
        cells = cells[inside]
        if not len(cells):
            continue
        fp, fw = element.face_rule_r(d, e, side, lev.r)
        fqw = fw * np.prod(np.delete(h, e) / 2.0)
        fv, fg = element.q_basis(lev.r, fp)
        grad = fg * (2.0 / h)                                    # (nq, nloc, d)
        fpb = element.pdisc_basis(lev.r, fp)
        nrm = np.zeros(d)
        nrm[e] = 1.0 if side else -1.0
        for a in range(k + 1):
            xb = X.reshape(k + 1, lev.R + lev.S)[a]
            vel = xb[:lev.R].reshape(lev.n_nodes, d)[lev.cell_nodes[cells]]       # (nc, nloc, d)
            pres = xb[lev.R:].reshape(lev.n_cells, lev.Shat)[cells]                # (nc, dim P)
            gv = np.einsum("qie,kic->kqce", grad, vel)           # d v_c / d x_e at face points
            pq = np.einsum("qm,km->kq", fpb, pres)
            trac = nu * np.einsum("kqce,e->kqc", gv, nrm) - pq[:, :, None] * nrm[None, None, :]
            out[a] -= np.einsum("q,kqc->c", fqw, trac)
    return out


def coefficients(forces: np.ndarray, u_mean: float, diameter: float) -> np.ndarray:
    """(c_D, c_L) = 2 F / (U_mean^2 D) for rho = 1."""
    return 2.0 * np.asarray(forces) / (u_mean ** 2 * diameter)
