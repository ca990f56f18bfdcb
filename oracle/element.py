"""Reference element of the inf-sup stable pair (Q2)^d x P1disc (oracle; test infrastructure only).

Sec. 2 builds V_h x Q_h on (Q_r)^d x P_{r-1}^disc; the hot path uses r = 2.
On the reference cell [-1, 1]^d:

* Q2: tensor products of the 1D Lagrange polynomials at {-1, 0, 1}; local node
  (l_x, l_y[, l_z]) in {0,1,2}^d has local number l_x + 3 l_y + 9 l_z;
* P1disc: {1, xi_1, ..., xi_d} in the cell's reference coordinates, so the
  first coefficient is the cell mean (reading of the unstated scaling);
* 3-point Gauss-Legendre rule per direction (exact to degree 5).
"""
from __future__ import annotations

import itertools

import numpy as np

GAUSS_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
GAUSS_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def lagrange1d(x) -> np.ndarray:
    """Values of the 1D Q2 Lagrange polynomials at nodes -1, 0, 1; shape (len(x), 3)."""
    x = np.asarray(x, float)
    return np.stack([x * (x - 1.0) / 2.0, 1.0 - x * x, x * (x + 1.0) / 2.0], axis=-1)


def lagrange1d_deriv(x) -> np.ndarray:
    x = np.asarray(x, float)
    return np.stack([x - 0.5, -2.0 * x, x + 0.5], axis=-1)


def local_nodes(dim: int) -> np.ndarray:
    """Local node multi-indices (n_loc, dim) with x fastest."""
    return np.array([idx[::-1] for idx in itertools.product(range(3), repeat=dim)])


def q2_basis(points: np.ndarray):
    """Q2 basis values (npts, 3^d) and reference gradients (npts, 3^d, d) at `points` (npts, d)."""
    points = np.atleast_2d(points)
    dim = points.shape[1]
    nodes = local_nodes(dim)
    v1 = lagrange1d(points)          # (npts, d, 3)
    d1 = lagrange1d_deriv(points)    # (npts, d, 3)
    npts = points.shape[0]
    vals = np.ones((npts, len(nodes)))
    grads = np.ones((npts, len(nodes), dim))
    for i, l in enumerate(nodes):
        for e in range(dim):
            vals[:, i] *= v1[:, e, l[e]]
            for g in range(dim):
                grads[:, i, g] *= d1[:, e, l[e]] if g == e else v1[:, e, l[e]]
    return vals, grads


def p1disc_basis(points: np.ndarray) -> np.ndarray:
    """P1disc basis {1, xi_1, .., xi_d} at `points`; shape (npts, d+1)."""
    points = np.atleast_2d(points)
    return np.concatenate([np.ones((points.shape[0], 1)), points], axis=1)


def cell_rule(dim: int):
    """Tensor Gauss rule on [-1,1]^d: points (3^d, d), weights (3^d,)."""
    idx = local_nodes(dim)
    return GAUSS_X[idx], np.prod(GAUSS_W[idx], axis=1)


def face_rule(dim: int, direction: int, side: int):
    """Gauss rule on the face xi_direction = -1 (side 0) or +1 (side 1) of [-1,1]^d."""
    if dim == 1:
        return np.array([[-1.0 if side == 0 else 1.0]]), np.array([1.0])
    idx = local_nodes(dim - 1)
    pts_f = GAUSS_X[idx]
    w = np.prod(GAUSS_W[idx], axis=1)
    pts = np.insert(pts_f, direction, -1.0 if side == 0 else 1.0, axis=1)
    return pts, w
