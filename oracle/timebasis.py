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


def radau_nodes(k: int) -> np.ndarray:
    """Right Gauss-Radau nodes on [0, 1] (k+1 points, the last one is 1)."""
    coef = np.zeros(k + 2)
    coef[k] = 1.0
    coef[k + 1] = -1.0
    x = np.sort(np.real(L.legroots(coef)))
    x[-1] = 1.0  # the root x = 1 is exact
    return (x + 1.0) / 2.0


def lagrange_values(nodes: np.ndarray, s) -> np.ndarray:
    """chi_a(s) in product form; shape (len(s), len(nodes))."""
    s = np.atleast_1d(np.asarray(s, float))
    out = np.ones((len(s), len(nodes)))
    for a, ca in enumerate(nodes):
        for b, cb in enumerate(nodes):
            if b != a:
                out[:, a] *= (s - cb) / (ca - cb)
    return out


def lagrange_derivatives(nodes: np.ndarray, s) -> np.ndarray:
    """chi_a'(s) = sum_{m != a} 1/(c_a - c_m) prod_{l != a, m} (s - c_l)/(c_a - c_l); shape (len(s), n)."""
    s = np.atleast_1d(np.asarray(s, float))
    n = len(nodes)
    out = np.zeros((len(s), n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            term = np.full(len(s), 1.0 / (nodes[a] - nodes[m]))
            for l in range(n):
                if l != a and l != m:
                    term *= (s - nodes[l]) / (nodes[a] - nodes[l])
            out[:, a] += term
    return out


def _gauss01(k: int):
    """(k+1)-point Gauss-Legendre rule on [0, 1] (exact to degree 2k+1)."""
    x, w = L.leggauss(k + 1)
    return (x + 1.0) / 2.0, w / 2.0


def radau_weights(k: int) -> np.ndarray:
    """w_a = int_0^1 chi_a(s) ds."""
    q, qw = _gauss01(k)
    return qw @ lagrange_values(radau_nodes(k), q)


def time_matrix(k: int) -> np.ndarray:
    """T_ab = int_0^1 chi_b' chi_a ds + chi_a(0) chi_b(0) (row a = test, column b = trial).

    The integrand has degree 2k - 1, so the (k+1)-point Gauss rule is exact; the
    Lagrange polynomials are evaluated in product form (a monomial expansion loses
    about 1e-12 relative accuracy at k = 4)."""
    nodes = radau_nodes(k)
    q, qw = _gauss01(k)
    chi = lagrange_values(nodes, q)
    dchi = lagrange_derivatives(nodes, q)
    j0 = lagrange_values(nodes, 0.0)[0]
    return np.einsum("q,qa,qb->ab", qw, chi, dchi) + np.outer(j0, j0)


def jump_vector(k: int) -> np.ndarray:
    """chi_a(0): the coefficient of the previous slab's end value in the jump term."""
    return lagrange_values(radau_nodes(k), 0.0)[0]


def eval_basis(k: int, s) -> np.ndarray:
    """chi_a(s) for all a, s in [0, 1]; shape (len(s), k+1)."""
    return lagrange_values(radau_nodes(k), s)
