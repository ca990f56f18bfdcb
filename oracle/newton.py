"""Nonlinear slab residual, damped Newton and time marching (oracle; test infrastructure only).

Sec. 3, Eq. (3.2): the slab problem of Eq. (2.2) is F_n(X_n) = 0.  With the
Radau rule in time (reading A2) the convection term ((v.grad)v, psi) of A_h at
Radau node a is the Oseen convection with w = v_a applied to v_a, so

    F_n(X) = J_Oseen(w = v(X)) X - b,
    b_a    = tau w_a [ (f_a, psi) + B_GammaD(g_a, (psi, xi)) ] + chi_a(0) M v_prev,

and the Newton Jacobian of Eq. (3.3) is the Jacobian with the Newton term at
w = v(X).  Sec. 3 solves J_n(X^m) C^m = -F(X^m) by a damped Newton method
(the damping rule is not stated; reading: halve lambda from 1 until
||F(X + lambda C)|| < (1 - 1e-4 lambda) ||F(X)||, lambda >= 1/16, else take
1/16), each linear system by the GMRES-GMG solver.  Data f, g and the
previous slab's end value are Q2 nodal fields (their interpolants enter the
integrals).
"""
from __future__ import annotations

import numpy as np

from . import assemble, element, fgmres, mesh, multigrid, timebasis


def velocity_part(lev, X: np.ndarray) -> np.ndarray:
    """(k+1, R) nodal velocities of a C-ABI vector."""
    xb = X.reshape(lev.k + 1, lev.R + lev.S)
    return np.ascontiguousarray(xb[:, :lev.R])


def end_value(lev, X: np.ndarray) -> np.ndarray:
    """v(t_n): the velocity at the last Radau node (right Radau: c_k = 1)."""
    return velocity_part(lev, X)[-1].copy()


def rhs_nodal(lev, f_nodal, g_nodal, v_prev, nu: float, tau: float,
              gamma1=assemble.GAMMA1, gamma2=assemble.GAMMA2) -> np.ndarray:
    """Right-hand side of Eq. (2.2) for Q2 nodal data (k+1, R) (None = 0) and v_prev (R,) (None = 0)."""
    d, k = lev.dim, lev.k
    h = np.asarray(lev.h)
    wts = timebasis.radau_weights(k)
    jump = timebasis.jump_vector(k)
    mmat = assemble.mass_matrix(lev)
    b = np.zeros(lev.N)
    for a in range(k + 1):
        s = tau * wts[a]
        blk = a * (lev.R + lev.S)
        vel = np.zeros(lev.R)
        pres = np.zeros(lev.S)
        if f_nodal is not None:
            vel += s * (mmat @ f_nodal[a])                       # (f_h, psi_i) = M f
        if v_prev is not None:
            vel += jump[a] * (mmat @ v_prev)
        if g_nodal is not None:
            gn = g_nodal[a].reshape(lev.n_nodes, d)
            vloc = np.zeros((lev.n_nodes, d))
            ploc = np.zeros((lev.n_cells, lev.Shat))
            for e, side, cells in lev.dirichlet_faces():
                fp, fw = element.face_rule_r(d, e, side, lev.r)
                fqw = fw * np.prod(np.delete(h, e) / 2.0)
                fv, fg = element.q_basis(lev.r, fp)
                nrm = np.zeros(d)
                nrm[e] = 1.0 if side == 1 else -1.0
                dn = (fg * (2.0 / h)) @ nrm
                fpb = element.pdisc_basis(lev.r, fp)
                gq = np.einsum("qj,kjc->kqc", fv, gn[lev.cell_nodes[cells]])   # g_h at face points
                gnq = gq @ nrm
                lv = (-nu * np.einsum("q,qi,kqc->kic", fqw, dn, gq)
                      + gamma1 * nu / h[e] * np.einsum("q,qi,kqc->kic", fqw, fv, gq)
                      + gamma2 / h[e] * np.einsum("q,qi,kq,c->kic", fqw, fv, gnq, nrm))
                np.add.at(vloc, lev.cell_nodes[cells], lv)
                ploc[cells] += -np.einsum("q,qm,kq->km", fqw, fpb, gnq)
            vel += s * vloc.ravel()
            pres += s * ploc.ravel()
        b[blk:blk + lev.R] += vel
        b[blk + lev.R:blk + lev.R + lev.S] += pres
    return b


def residual(lev, X: np.ndarray, b: np.ndarray, nu: float, tau: float) -> np.ndarray:
    """F_n(X) = J_Oseen(w = v(X)) X - b."""
    jac = assemble.jacobian(lev, velocity_part(lev, X), nu, tau, newton=False)
    return jac @ X - b


def newton_slab(spec, k, nu, tau, X0, b, rtol=1e-8, atol=0.0, maxit=20, gmres_rtol=1e-8, nu1=2, nu2=2,
                lam_min=1.0 / 16.0, lambdas=None):
    """Damped Newton for F_n(X) = 0; returns (X, Newton steps, total GMRES iterations, ||F|| history).

    `lambdas`, if a list, receives the damping factor accepted at each step."""
    lev = mesh.Level(spec, spec.n_levels - 1, k)
    X = np.array(X0, dtype=float, copy=True)
    F = residual(lev, X, b, nu, tau)
    hist = [np.linalg.norm(F)]
    tol = max(rtol * hist[0], atol)
    its_total = 0
    steps = 0
    while hist[-1] > tol and steps < maxit:
        h = multigrid.Hierarchy(spec, k, nu, tau, velocity_part(lev, X), newton=True, nu1=nu1, nu2=nu2)
        C, its, rel, ok = fgmres.fgmres(h.apply, h.vcycle, -F, rtol=gmres_rtol)
        its_total += its
        lam = 1.0
        while True:
            Xt = X + lam * C
            Ft = residual(lev, Xt, b, nu, tau)
            if np.linalg.norm(Ft) < (1.0 - 1e-4 * lam) * hist[-1] or lam <= lam_min:
                break
            lam *= 0.5
        X, F = Xt, Ft
        hist.append(np.linalg.norm(F))
        if lambdas is not None:
            lambdas.append(lam)
        steps += 1
    return X, steps, its_total, hist
