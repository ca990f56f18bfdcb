"""Right-preconditioned flexible GMRES (oracle; test infrastructure only).

Sec. 3 solves J C = -F by GMRES iterations [Saad 2003] preconditioned by one
V-cycle.  Reading: flexible GMRES(m) with right preconditioning (Saad,
Iterative Methods for Sparse Linear Systems, 2nd ed., Sec. 9.4.1), modified
Gram-Schmidt Arnoldi, Givens rotations, restart length m = 30, stopping when
||b - J x|| <= max(rtol ||b||, atol); the true residual is recomputed before
the method reports convergence.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_a, precond, b: np.ndarray, x0: np.ndarray | None = None, restart: int = 30,
           rtol: float = 1e-8, atol: float = 0.0, maxit: int = 500):
    """Returns (x, total inner iterations, final ||b - A x|| / ||b||, converged flag)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float, copy=True)
    bnorm = np.linalg.norm(b)
    tol = max(rtol * bnorm, atol)
    its = 0
    while True:
        r = b - apply_a(x)
        beta = np.linalg.norm(r)
        if beta <= tol or its >= maxit or bnorm == 0.0:
            rel = beta / bnorm if bnorm > 0 else 0.0
            return x, its, rel, beta <= tol
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_a(Z[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.hypot(H[j, j], H[j + 1, j])         # new rotation
            cs[j] = H[j, j] / rho
            sn[j] = H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            if abs(g[j + 1]) <= tol or its >= maxit or H[j, j] == 0.0:
                break
        # y = H^{-1} g by back substitution, x += Z y
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_end], y[i + 1:j_end])) / H[i, i]
        x = x + Z[:j_end].T @ y
