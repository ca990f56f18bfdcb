"""Grid transfer between nested levels (oracle; test infrastructure only).

The paper uses a geometric V-cycle on nested meshes (Sec. 2: T_0 .. T_L with
h_l = gamma h_{l-1}; Sec. 3) but does not state the transfer operators.
Reading: the canonical ones of nested conforming spaces.  The prolongation P
maps the coefficients of a coarse finite element function to the coefficients
of the same function on the fine mesh (Q2: its values at the fine nodes;
P1disc: its P1 expansion on each child cell); the restriction is P^T.  Time
nodes are not coarsened: P acts identically on every Radau node block.  With an
obstacle the spaces are those of the fluid domain: P is zero on the fine unknowns
outside it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import element


def _coarse_cell_and_ref(coarse, xyz: np.ndarray):
    """Coarse cell containing each point and the point's reference coordinates in it."""
    lo = np.asarray(coarse.spec.lo)
    h = np.asarray(coarse.h)
    u = (xyz - lo) / h
    ci = np.clip(np.floor(u + 1e-12).astype(np.int64), 0, np.asarray(coarse.cells) - 1)
    ref = 2.0 * (u - ci) - 1.0
    cell = np.zeros(len(xyz), dtype=np.int64)
    stride = 1
    for e in range(coarse.dim):
        cell += ci[:, e] * stride
        stride *= coarse.cells[e]
    return cell, ref


def prolongation(coarse, fine) -> sp.csr_matrix:
    """P: coarse C-ABI vector -> fine C-ABI vector (all k+1 time nodes)."""
    d, k = fine.dim, fine.k
    # velocity: evaluate the coarse Q2 functions at the fine nodes
    fx = fine.node_coords()
    cell, ref = _coarse_cell_and_ref(coarse, fx)
    vals, _ = element.q_basis(fine.r, ref)                 # (n_fine_nodes, nloc)
    cn = coarse.cell_nodes[cell]                           # (n_fine_nodes, nloc)
    vr, vc, vv = [], [], []
    for c in range(d):
        vr.append(np.repeat(np.arange(fine.n_nodes) * d + c, cn.shape[1]))
        vc.append((cn * d + c).ravel())
        vv.append(vals.ravel())
    pv = sp.coo_matrix((np.concatenate(vv), (np.concatenate(vr), np.concatenate(vc))),
                       shape=(fine.R, coarse.R)).tocsr()
    pv.sum_duplicates()
    if fine.r != 2:
        pp = _pdisc_prolongation(coarse, fine)
        blk = sp.block_diag([pv, pp], format="csr")
        return _mask_dead(fine, sp.block_diag([blk] * (k + 1), format="csr"))
    # pressure: fine P1 coefficients of the coarse P1 function on each child
    centres = fine.cell_centres()
    h = np.asarray(fine.h)
    pr, pc, pval = [], [], []
    ccell, cref0 = _coarse_cell_and_ref(coarse, centres)
    base0 = element.p1disc_basis(cref0)                     # coarse basis at the child centre
    for m in range(d + 1):
        # fine coefficient 0: value at the child centre
        pr.append(np.arange(fine.n_cells) * (d + 1))
        pc.append(ccell * (d + 1) + m)
        pval.append(base0[:, m])
        for e in range(d):
            # fine coefficient e+1: change of the (linear) coarse function between xi_f = 0 and xi_f = e_e
            shifted = centres.copy()
            shifted[:, e] += h[e] / 2.0
            _, cref1 = _coarse_cell_and_ref_fixed(coarse, shifted, ccell)
            base1 = element.p1disc_basis(cref1)
            pr.append(np.arange(fine.n_cells) * (d + 1) + e + 1)
            pc.append(ccell * (d + 1) + m)
            pval.append(base1[:, m] - base0[:, m])
    pp = sp.coo_matrix((np.concatenate(pval), (np.concatenate(pr), np.concatenate(pc))),
                       shape=(fine.S, coarse.S)).tocsr()
    pp.eliminate_zeros()
    blk = sp.block_diag([pv, pp], format="csr")
    return _mask_dead(fine, sp.block_diag([blk] * (k + 1), format="csr"))


def _pdisc_prolongation(coarse, fine) -> sp.csr_matrix:
    """P_{r-1}^disc: the coefficients of the coarse cell's polynomial on each child cell (the
    space is invariant under the child's affine map, so the fine coefficients solve the
    interpolation at the child's Gauss points exactly)."""
    d, r, sh = fine.dim, fine.r, fine.Shat
    pts, _ = element.cell_rule_r(d, r)                       # child reference points (more than dim P)
    bf = element.pdisc_basis(r, pts)                         # (nq, sh)
    rows, cols, vals = [], [], []
    for child in range(fine.n_cells):
        ci = fine.cell_idx[child]
        cc = ci // 2
        cell_c = int(sum(cc[e] * int(np.prod(coarse.cells[:e])) for e in range(d)))
        off = ci - 2 * cc                                    # 0 or 1 per direction
        ref_c = (pts + 1.0) / 2.0 + off[None, :] - 1.0       # child point in the coarse cell
        bc = element.pdisc_basis(r, ref_c)                   # (nq, sh)
        m = np.linalg.lstsq(bf, bc, rcond=None)[0]           # fine coefficients of each coarse basis fn
        for i in range(sh):
            for j in range(sh):
                if abs(m[i, j]) > 1e-15:
                    rows.append(child * sh + i)
                    cols.append(cell_c * sh + j)
                    vals.append(m[i, j])
    return sp.coo_matrix((vals, (rows, cols)), shape=(fine.S, coarse.S)).tocsr()


def _mask_dead(fine, out):
    if fine.masked.any():
        # obstacle domain: the fine unknowns without an equation (outside the domain) are not
        # part of the nested space; P sets them to zero, so R = P^T never carries their residual
        # into the coarse unknowns of the obstacle's boundary
        from .assemble import dead_dofs
        keep = np.ones(fine.N)
        keep[dead_dofs(fine)] = 0.0
        out = sp.diags(keep) @ out
        out = sp.csr_matrix(out)
        out.eliminate_zeros()
    return out


def _coarse_cell_and_ref_fixed(coarse, xyz, cell):
    """Reference coordinates of points in given coarse cells (the points may lie on the cell boundary)."""
    lo = np.asarray(coarse.spec.lo)
    h = np.asarray(coarse.h)
    ci = coarse.cell_idx[cell]
    u = (xyz - lo) / h
    return cell, 2.0 * (u - ci) - 1.0
