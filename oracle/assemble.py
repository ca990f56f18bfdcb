"""Jacobian of the space-time slab problem (oracle; test infrastructure only).

Follows Sec. 2 and Sec. 3 of the paper:

* A_h (Sec. 2) gives, for the linearisation velocity w at Radau node a:
  convection ((w . grad) v, psi), for Newton also ((v . grad) w, psi),
  viscosity nu (grad v, grad psi), pressure -(p, div psi), divergence
  (div v, xi), the consistency term -<nu grad v . n - p n, psi> on Gamma_D and
  B_GammaD(v, (psi, xi)) of Eq. (2.1) with gamma1 = gamma2 = 35;
* Eq. (2.2) integrates A_h over I_n and adds the time derivative and the jump;
* Eq. (3.3) arranges the Jacobian in (k+1) x (k+1) saddle-point blocks
  J_ab = [[D_ab, B_ab^T], [B_ab, 0]] with D_ab and B_ab^T as printed after it.

Readings (listed with the others in the design notes):
* row = test function (a, i), column = trial function (b, j);
* all time integrals use the (k+1)-point Radau rule, so the spatial parts of
  D_ab and B_ab vanish for a != b and carry the factor tau * w_a;
* the time derivative plus jump gives T_ab * M (timebasis.time_matrix);
* Nitsche signs follow A_h and B_GammaD (both boundary terms with minus), the
  pressure blocks follow A_h: -(p, div psi) + <p n, psi> and
  (div v, xi) - <v . n, xi>; h = |K| / |F|;
* the spatial rule is the 3^d-point Gauss rule for every term.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import element, timebasis

GAMMA1 = 35.0
GAMMA2 = 35.0


class CellOperators:
    """Per-cell spatial matrices of one level for the linearisation velocity w."""

    def __init__(self, lev, w: np.ndarray, nu: float, newton: bool, gamma1=GAMMA1, gamma2=GAMMA2):
        d = lev.dim
        self.lev = lev
        h = np.asarray(lev.h)
        r = lev.r
        pts, wts = element.cell_rule_r(d, r)
        det = np.prod(h / 2.0)
        vals, gref = element.q_basis(r, pts)
        gphys = gref * (2.0 / h)                     # (nq, nloc, d)
        pb = element.pdisc_basis(r, pts)             # (nq, dim P)
        qw = wts * det
        nloc = lev.n_loc_nodes
        self.mass = np.einsum("q,qi,qj->ij", qw, vals, vals)
        self.stiff = np.einsum("q,qie,qje->ij", qw, gphys, gphys)
        # (div psi_{j,e}, xi_m): shape (m, j, e)
        self.div = np.einsum("q,qje,qm->mje", qw, gphys, pb)

        k = lev.k
        nc = lev.n_cells
        # w at cell nodes, per time node: (k+1, ncells, nloc, d)
        wn = w.reshape(k + 1, lev.n_nodes, d)
        wc = wn[:, lev.cell_nodes, :]
        wq = np.einsum("qi,akid->akqd", vals, wc)                 # w at quadrature points
        gw = np.einsum("qie,akic->akqce", gphys, wc)              # d w_c / d x_e
        # convection (w . grad phi_j, phi_i): (k+1, ncells, i, j)
        self.conv = np.einsum("q,akqe,qje,qi->akij", qw, wq, gphys, vals)
        if newton:
            # ((phi_j e_e) . grad) w, phi_i e_c) = phi_j d_e w_c phi_i: (k+1, ncells, i, c, j, e)
            self.newt = np.einsum("q,qi,qj,akqce->akicje", qw, vals, vals, gw)
        else:
            self.newt = None

        # Nitsche face terms per cell: velocity-velocity (ncells, i, c, j, e), pressure (ncells, i, c, m)
        vv = np.zeros((nc, nloc, d, nloc, d))
        vp = np.zeros((nc, nloc, d, lev.Shat))
        # Dirichlet faces: the domain's (a do-nothing face is the natural condition of A_h and
        # carries no boundary term) and those of an obstacle
        for e, side, cells in lev.dirichlet_faces():
            fp, fw = element.face_rule_r(d, e, side, r)
            fdet = np.prod(np.delete(h, e) / 2.0)
            fqw = fw * fdet
            fv, fg = element.q_basis(r, fp)
            fgp = fg * (2.0 / h)
            nrm = np.zeros(d)
            nrm[e] = 1.0 if side == 1 else -1.0
            dn = fgp @ nrm                                    # normal derivative (nf, nloc)
            hf = h[e]
            fpb = element.pdisc_basis(r, fp)
            consist = -nu * np.einsum("q,qj,qi->ij", fqw, dn, fv)     # -<nu d_n phi_j, phi_i>
            symm = -nu * np.einsum("q,qj,qi->ij", fqw, fv, dn)        # -<phi_j, nu d_n phi_i>
            pen1 = gamma1 * nu / hf * np.einsum("q,qj,qi->ij", fqw, fv, fv)
            mass_f = np.einsum("q,qj,qi->ij", fqw, fv, fv)
            blk = np.zeros((nloc, d, nloc, d))
            for c in range(d):
                blk[:, c, :, c] += consist + symm + pen1
            # gamma2 h^-1 <phi_j n_e, phi_i n_c>
            blk += gamma2 / hf * np.einsum("ij,c,e->icje", mass_f, nrm, nrm)
            vv[cells] += blk
            # <xi_m n, psi_i> in the velocity rows
            vp[cells] += np.einsum("q,qi,qm,c->icm", fqw, fv, fpb, nrm)
        self.face_vv = vv
        self.face_vp = vp


def element_matrices(lev, w: np.ndarray, nu: float, tau: float, newton: bool,
                     gamma1=GAMMA1, gamma2=GAMMA2) -> np.ndarray:
    """Space-time element matrices (ncells, n_patch, n_patch) in the local order of mesh.Level."""
    ops = CellOperators(lev, w, nu, newton, gamma1, gamma2)
    d, k, nloc = lev.dim, lev.k, lev.n_loc_nodes
    nc = lev.n_cells
    tmat = timebasis.time_matrix(k)
    wts = timebasis.radau_weights(k)
    eye = np.eye(d)
    out = np.zeros((nc, lev.n_patch, lev.n_patch))
    blk = lev.Rhat + lev.Shat
    for a in range(k + 1):
        ra = slice(a * blk, a * blk + lev.Rhat)              # velocity rows of time node a
        pa = slice(a * blk + lev.Rhat, (a + 1) * blk)        # pressure rows of time node a
        for b in range(k + 1):
            cb = slice(b * blk, b * blk + lev.Rhat)
            # time derivative + jump: T_ab M (component diagonal)
            out[:, ra, cb] += tmat[a, b] * np.einsum("ij,ce->icje", ops.mass, eye).reshape(lev.Rhat, lev.Rhat)
        s = tau * wts[a]
        spatial = np.einsum("kij,ce->kicje", ops.conv[a] + nu * ops.stiff[None], eye)
        if ops.newt is not None:
            spatial = spatial + ops.newt[a]
        spatial = spatial + ops.face_vv
        out[:, ra, ra] += s * spatial.reshape(nc, lev.Rhat, lev.Rhat)
        # velocity rows, pressure columns: -(xi_m, div psi_i) + <xi_m n, psi_i>
        vp = -np.transpose(ops.div, (1, 2, 0))[None] + ops.face_vp          # (nc, i, c, m)
        out[:, ra, pa] += s * vp.reshape(nc, lev.Rhat, lev.Shat)
        # pressure rows, velocity columns: (div psi_j, xi_m) - <psi_j . n, xi_m>
        pv = ops.div[None] - np.transpose(ops.face_vp, (0, 3, 1, 2))        # (nc, m, j, e)
        out[:, pa, ra] += s * pv.reshape(nc, lev.Shat, lev.Rhat)
    out[lev.masked] = 0.0            # cells removed by an obstacle carry no element matrices
    return out


def dead_dofs(lev) -> np.ndarray:
    """Unknowns without an equation in the obstacle domain: the velocity at Q2 nodes of removed
    cells only and the pressure of removed cells, every Radau node (C-ABI numbers)."""
    if not lev.masked.any():
        return np.zeros(0, dtype=np.int64)
    out = []
    cells = np.nonzero(lev.masked)[0]
    for a in range(lev.k + 1):
        for c in range(lev.dim):
            out.append(lev.vel_index(a, lev.dead_nodes, c))
        for m in range(lev.Shat):
            out.append(lev.pres_index(a, cells, m))
    return np.sort(np.concatenate(out))


def jacobian(lev, w: np.ndarray, nu: float, tau: float, newton: bool,
             gamma1=GAMMA1, gamma2=GAMMA2) -> sp.csr_matrix:
    """Global Jacobian J of Eq. (3.3) on one level, CSR in the C-ABI order."""
    emat = element_matrices(lev, w, nu, tau, newton, gamma1, gamma2)
    rows = np.broadcast_to(lev.dof[:, :, None], emat.shape).ravel()
    cols = np.broadcast_to(lev.dof[:, None, :], emat.shape).ravel()
    jac = sp.coo_matrix((emat.ravel(), (rows, cols)), shape=(lev.N, lev.N)).tocsr()
    dead = dead_dofs(lev)
    if len(dead):
        jac = jac + sp.csr_matrix((np.ones(len(dead)), (dead, dead)), shape=(lev.N, lev.N))
    jac.sum_duplicates()
    jac.eliminate_zeros()
    return jac


def mass_matrix(lev) -> sp.csr_matrix:
    """Scalar-per-component velocity mass matrix on one time node block (R x R)."""
    d = lev.dim
    pts, wts = element.cell_rule_r(d, lev.r)
    vals, _ = element.q_basis(lev.r, pts)
    me = np.einsum("q,qi,qj->ij", wts * np.prod(np.asarray(lev.h) / 2.0), vals, vals)
    rows, cols, data = [], [], []
    cn = lev.cell_nodes[~lev.masked]                 # cells removed by an obstacle add nothing
    for c in range(d):
        ri = cn[:, :, None] * d + c
        ci = cn[:, None, :] * d + c
        rows.append(np.broadcast_to(ri, (len(cn),) + me.shape).ravel())
        cols.append(np.broadcast_to(ci, (len(cn),) + me.shape).ravel())
        data.append(np.broadcast_to(me, (len(cn),) + me.shape).ravel())
    return sp.coo_matrix((np.concatenate(data), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(lev.R, lev.R)).tocsr()


def rhs_linear(lev, f, g, v_prev, nu: float, tau: float, t0: float = 0.0,
               gamma1=GAMMA1, gamma2=GAMMA2) -> np.ndarray:
    """Right-hand side of Eq. (2.2) for given data.

    b_a = tau w_a [ (f(t_a), psi) + B_GammaD(g(t_a), (psi, xi)) ] + chi_a(0) M v_prev,
    with f(x, t), g(x, t) callables returning (npts, d) and v_prev the previous
    slab's end value as an R-vector (or None for zero).
    """
    d, k = lev.dim, lev.k
    h = np.asarray(lev.h)
    cn = timebasis.radau_nodes(k)
    wts = timebasis.radau_weights(k)
    jump = timebasis.jump_vector(k)
    b = np.zeros(lev.N)
    pts, qw = element.cell_rule_r(d, lev.r)
    det = np.prod(h / 2.0)
    vals, _ = element.q_basis(lev.r, pts)
    centres = lev.cell_centres()
    for a in range(k + 1):
        ta = t0 + tau * cn[a]
        s = tau * wts[a]
        xq = centres[:, None, :] + pts[None, :, :] * (h / 2.0)      # (nc, nq, d)
        fq = f(xq.reshape(-1, d), ta).reshape(lev.n_cells, -1, d)
        loc = np.einsum("q,qi,kqc->kic", qw * det, vals, fq)       # (nc, nloc, d)
        loc[lev.masked] = 0.0
        vel = np.zeros((lev.n_nodes, d))
        np.add.at(vel, lev.cell_nodes, loc)
        pres = np.zeros((lev.n_cells, lev.Shat))
        for e, side, cells in lev.dirichlet_faces():
            if g is None:
                continue
            fp, fw = element.face_rule_r(d, e, side, lev.r)
            fqw = fw * np.prod(np.delete(h, e) / 2.0)
            fv, fg = element.q_basis(lev.r, fp)
            nrm = np.zeros(d)
            nrm[e] = 1.0 if side == 1 else -1.0
            dn = (fg * (2.0 / h)) @ nrm
            fpb = element.pdisc_basis(lev.r, fp)
            xf = centres[cells][:, None, :] + fp[None] * (h / 2.0)
            gq = g(xf.reshape(-1, d), ta).reshape(len(cells), -1, d)
            gn = gq @ nrm
            lv = (-nu * np.einsum("q,qi,kqc->kic", fqw, dn, gq)
                  + gamma1 * nu / h[e] * np.einsum("q,qi,kqc->kic", fqw, fv, gq)
                  + gamma2 / h[e] * np.einsum("q,qi,kq,c->kic", fqw, fv, gn, nrm))
            np.add.at(vel, lev.cell_nodes[cells], lv)
            pres[cells] += -np.einsum("q,qm,kq->km", fqw, fpb, gn)
        blk = a * (lev.R + lev.S)
        b[blk:blk + lev.R] += s * vel.ravel()
        b[blk + lev.R:blk + lev.R + lev.S] += s * pres.ravel()
    if v_prev is not None:
        mv = mass_matrix(lev) @ v_prev
        for a in range(k + 1):
            blk = a * (lev.R + lev.S)
            b[blk:blk + lev.R] += jump[a] * mv
    return b
