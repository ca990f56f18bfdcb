"""Time basis of the dG(k) slab problem (oracle; test infrastructure only).

Sec. 3 of the paper represents the discrete solution on I_n = (t_{n-1}, t_n] in
the Lagrange basis {chi_{n,a}} at the k+1 Gauss-Radau points of I_n, and the
time derivative and the jump term of Eq. (2.2) act through that basis.  On the
reference interval [0, 1] (t = t_{n-1} + tau * s):

* right Radau nodes c_a: the roots of P_k - P_{k+1} on [-1, 1] mapped by
  s = (x + 1) / 2; they include s = 1 = t_n (reading: I_n is open on the left);
* weights w_a = int_0^1 chi_a(s) ds (interpolatory rule, exact to degree 2k);
* T_ab = int_0^1 chi_b'(s) chi_a(s) ds + chi_a(0) chi_b(0): the time-derivative
  plus jump part of D_ab, row = test index a, column = trial index b;
* jump vector chi_a(0): the weight of the previous slab's end value in row a.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L
from numpy.polynomial import polynomial as P


def radau_nodes(k: int) -> np.ndarray:
    """Right Gauss-Radau nodes on [0, 1] (k+1 points, the last one is 1)."""
    coef = np.zeros(k + 2)
    coef[k] = 1.0
    coef[k + 1] = -1.0
    x = np.sort(np.real(L.legroots(coef)))
    x[-1] = 1.0  # the root x = 1 is exact
    return (x + 1.0) / 2.0


def lagrange_polys(nodes: np.ndarray) -> list:
    """Power-series coefficients of the Lagrange polynomials chi_a at `nodes`."""
    polys = []
    for a, ca in enumerate(nodes):
        others = np.delete(nodes, a)
        num = P.polyfromroots(others) if len(others) else np.array([1.0])
        polys.append(num / np.prod(ca - others))
    return polys


def radau_weights(k: int) -> np.ndarray:
    chis = lagrange_polys(radau_nodes(k))
    return np.array([P.polyval(1.0, P.polyint(c)) - P.polyval(0.0, P.polyint(c)) for c in chis])


def time_matrix(k: int) -> np.ndarray:
    """T_ab = int_0^1 chi_b' chi_a ds + chi_a(0) chi_b(0) (row a = test, column b = trial)."""
    chis = lagrange_polys(radau_nodes(k))
    n = k + 1
    t = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            integrand = P.polymul(P.polyder(chis[b]), chis[a])
            anti = P.polyint(integrand)
            t[a, b] = P.polyval(1.0, anti) - P.polyval(0.0, anti) + P.polyval(0.0, chis[a]) * P.polyval(0.0, chis[b])
    return t


def jump_vector(k: int) -> np.ndarray:
    """chi_a(0): the coefficient of the previous slab's end value in the jump term."""
    return np.array([P.polyval(0.0, c) for c in lagrange_polys(radau_nodes(k))])


def eval_basis(k: int, s) -> np.ndarray:
    """chi_a(s) for all a, s in [0, 1]; shape (len(s), k+1)."""
    s = np.atleast_1d(np.asarray(s, float))
    return np.stack([P.polyval(s, c) for c in lagrange_polys(radau_nodes(k))], axis=1)
