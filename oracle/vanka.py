"""Local Vanka smoother (oracle; test infrastructure only).

Sec. 3, Eq. (3.4): S_K(d) = R_K d + omega J_K^{-1} R_K (b - J d), omega = 0.7,
where R_K gathers the (k+1)(R^+S^) values dof(K, .) and J_K is the restriction
of the assembled J to those rows and columns; the paper inverts J_K with LAPACK
(numpy.linalg.inv calls LAPACK getrf/getri here).

The smoothing loop (S0)-(S3) after Eq. (3.4), with d^0 given:
  for j = 1..J_max:
      p = 0, z = 0                                   (S0)
      for every cell K: y_K = S_K(d^{j-1})           (S1)
          z[dof(K, .)] += y_K ; p[dof(K, .)] += 1    (S2)
      d^j = z / p                                    (S3)
The paper remarks that this averaging is used instead of overwriting the
values successively.  The successive variant is provided as `sweep_coloured`:
cells are visited colour by colour, with the residual refreshed before each
colour (cells of one colour share no velocity DoF).
"""
from __future__ import annotations

import numpy as np


def patch_active(lev) -> np.ndarray:
    """(ncells, n_patch) bool: the local unknowns each patch smooths.  A cell of the fluid domain
    smooths all of its unknowns.  With an obstacle (cells removed from the mesh), a removed cell's
    patch holds only its unknowns without an equation (velocity at Q2 nodes of removed cells only,
    its pressure), whose rows are the identity: the paper's patches are the cells of the mesh, and
    the unknowns outside the domain are solved exactly in patches of their own."""
    act = np.ones((lev.n_cells, lev.n_patch), dtype=bool)
    if lev.masked.any():
        dead = np.zeros(lev.N, dtype=bool)
        from .assemble import dead_dofs
        dead[dead_dofs(lev)] = True
        act[lev.masked] = dead[lev.dof[lev.masked]]
    return act


def local_matrices(jac, lev) -> np.ndarray:
    """J_K = J[dof(K,.), dof(K,.)] for every cell: (ncells, n_patch, n_patch)."""
    out = np.zeros((lev.n_cells, lev.n_patch, lev.n_patch))
    csr = jac.tocsr()
    for cell in range(lev.n_cells):
        idx = lev.dof[cell]
        out[cell] = csr[idx][:, idx].toarray()
    return out


def local_inverses(jac, lev) -> np.ndarray:
    """J_K^{-1} for every cell via LAPACK (numpy.linalg.inv).  A removed cell's patch (see
    patch_active) acts on its identity rows only: its inverse is the projector onto them."""
    if not lev.masked.any():
        return np.linalg.inv(local_matrices(jac, lev))
    act = patch_active(lev)
    out = np.zeros((lev.n_cells, lev.n_patch, lev.n_patch))
    fluid = ~lev.masked
    out[fluid] = np.linalg.inv(local_matrices(jac, lev)[fluid])
    for cell in np.nonzero(lev.masked)[0]:
        out[cell] = np.diag(act[cell].astype(float))
    return out


def sweep_averaged(jac, lev, jinv, b, d, omega: float = 0.7, sweeps: int = 1) -> np.ndarray:
    """J_max = `sweeps` iterations of (S0)-(S3) starting from d^0 = d."""
    dof = lev.dof
    act = patch_active(lev).astype(float)
    d = np.array(d, dtype=float, copy=True)
    for _ in range(sweeps):
        p = np.zeros(lev.N)                                      # (S0)
        z = np.zeros(lev.N)
        r = b - jac @ d                                          # b - J d^{j-1}, shared by all K
        y = d[dof] + omega * np.einsum("kij,kj->ki", jinv, r[dof])   # (S1): S_K(d^{j-1})
        np.add.at(z, dof, y * act)                               # (S2), over each patch's unknowns
        np.add.at(p, dof, act)
        d = z / p                                                # (S3)
    return d


def sweep_coloured(jac, lev, jinv, b, d, omega: float = 0.7, sweeps: int = 1) -> np.ndarray:
    """Successive (multiplicative) variant: colour by colour, d <- d + omega E_K J_K^{-1} R_K (b - J d)."""
    dof = lev.dof
    d = np.array(d, dtype=float, copy=True)
    for _ in range(sweeps):
        for colour in range(2 ** lev.dim):
            cells = np.nonzero(lev.colour == colour)[0]
            r = b - jac @ d
            y = omega * np.einsum("kij,kj->ki", jinv[cells], r[dof[cells]])
            np.add.at(d, dof[cells], y)
    return d
