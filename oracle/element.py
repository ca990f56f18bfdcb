"""Reference element of the inf-sup stable pair (Q_r)^d x P_{r-1}^disc (oracle; test infrastructure only).

Sec. 2 builds V_h x Q_h on (Q_r)^d x P_{r-1}^disc; the 3D experiment of Sec. 4 uses r = 2, the 2D
one r = 4.  On the reference cell [-1, 1]^d:

* Q_r: tensor products of the 1D Lagrange polynomials at the r + 1 equidistant points
  -1 + 2 l / r; local node (l_x, l_y[, l_z]) in {0..r}^d has local number
  l_x + (r+1) l_y + (r+1)^2 l_z (r = 2: {-1, 0, 1}, l_x + 3 l_y + 9 l_z);
* P_{r-1}^disc: the monomials xi^a eta^b (zeta^c) of total degree <= r - 1 in the cell's reference
  coordinates, by degree and then with the x exponent falling (r = 2: {1, xi_1, ..., xi_d}, so the
  first coefficient is the cell mean: reading of the unstated scaling);
* the (r+1)-point Gauss-Legendre rule per direction (exact to degree 2r + 1; r = 2: 3 points).
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


# ---------------------------------------------------------------- general order r (r = 2 above)
def gauss_rule_1d(r: int):
    """(r+1)-point Gauss-Legendre points and weights on [-1, 1] (r = 2: the constants above;
    r = 4: the closed form, points +-sqrt(5 -+ 2 sqrt(10/7)) / 3 and 0, weights
    (322 +- 13 sqrt(70)) / 900 and 128/225)."""
    if r == 2:
        return GAUSS_X, GAUSS_W
    if r == 4:
        a = np.sqrt(5.0 - 2.0 * np.sqrt(10.0 / 7.0)) / 3.0
        b = np.sqrt(5.0 + 2.0 * np.sqrt(10.0 / 7.0)) / 3.0
        wa = (322.0 + 13.0 * np.sqrt(70.0)) / 900.0
        wb = (322.0 - 13.0 * np.sqrt(70.0)) / 900.0
        return np.array([-b, -a, 0.0, a, b]), np.array([wb, wa, 128.0 / 225.0, wa, wb])
    x, w = np.polynomial.legendre.leggauss(r + 1)
    return x, w


def local_nodes_r(dim: int, r: int) -> np.ndarray:
    """Local node multi-indices (n_loc, dim) of Q_r with x fastest."""
    if r == 2:
        return local_nodes(dim)
    return np.array([idx[::-1] for idx in itertools.product(range(r + 1), repeat=dim)])


def lagrange1d_r(r: int, x):
    """Values and derivatives of the 1D Q_r Lagrange polynomials at the equidistant nodes;
    shapes (..., r+1)."""
    x = np.asarray(x, float)
    if r == 2:
        return lagrange1d(x), lagrange1d_deriv(x)
    nodes = -1.0 + 2.0 * np.arange(r + 1) / r
    vals = np.ones(x.shape + (r + 1,))
    ders = np.zeros(x.shape + (r + 1,))
    for l in range(r + 1):
        others = [m for m in range(r + 1) if m != l]
        den = np.prod([nodes[l] - nodes[m] for m in others])
        for m in others:
            vals[..., l] *= (x - nodes[m])
        # derivative of the product: sum over the factor left out
        for q in others:
            term = np.ones(x.shape)
            for m in others:
                if m != q:
                    term = term * (x - nodes[m])
            ders[..., l] += term
        vals[..., l] /= den
        ders[..., l] /= den
    return vals, ders


def q_basis(r: int, points: np.ndarray):
    """Q_r basis values (npts, (r+1)^d) and reference gradients (npts, (r+1)^d, d)."""
    if r == 2:
        return q2_basis(points)
    points = np.atleast_2d(points)
    dim = points.shape[1]
    nodes = local_nodes_r(dim, r)
    v1, d1 = lagrange1d_r(r, points)          # (npts, d, r+1)
    npts = points.shape[0]
    vals = np.ones((npts, len(nodes)))
    grads = np.ones((npts, len(nodes), dim))
    for i, l in enumerate(nodes):
        for e in range(dim):
            vals[:, i] *= v1[:, e, l[e]]
            for g in range(dim):
                grads[:, i, g] *= d1[:, e, l[e]] if g == e else v1[:, e, l[e]]
    return vals, grads


def pdisc_exponents(r: int, dim: int) -> list:
    """Exponents of the P_{r-1}^disc monomials: by total degree, then the x exponent falling."""
    out = []
    for deg in range(r):
        for a in itertools.product(range(deg + 1), repeat=dim):
            if sum(a) == deg:
                out.append(a)
    out_sorted = []
    for deg in range(r):
        group = [a for a in out if sum(a) == deg]
        group.sort(key=lambda a: tuple(-v for v in a))
        out_sorted += group
    return out_sorted


def pdisc_basis(r: int, points: np.ndarray) -> np.ndarray:
    """P_{r-1}^disc basis at `points`; shape (npts, dim P_{r-1})."""
    if r == 2:
        return p1disc_basis(points)
    points = np.atleast_2d(points)
    ex = pdisc_exponents(r, points.shape[1])
    return np.stack([np.prod(points ** np.asarray(a)[None, :], axis=1) for a in ex], axis=1)


def cell_rule_r(dim: int, r: int):
    """Tensor (r+1)-point Gauss rule on [-1,1]^d."""
    if r == 2:
        return cell_rule(dim)
    x, w = gauss_rule_1d(r)
    idx = local_nodes_r(dim, r)
    return x[idx], np.prod(w[idx], axis=1)


def face_rule_r(dim: int, direction: int, side: int, r: int):
    """(r+1)-point Gauss rule on the face xi_direction = -1 (side 0) or +1 (side 1)."""
    if r == 2:
        return face_rule(dim, direction, side)
    x, w = gauss_rule_1d(r)
    idx = local_nodes_r(dim - 1, r)
    pts_f = x[idx]
    wf = np.prod(w[idx], axis=1)
    pts = np.insert(pts_f, direction, -1.0 if side == 0 else 1.0, axis=1)
    return pts, wf
