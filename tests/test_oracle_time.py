"""Pins of the oracle's time basis (Sec. 3: Lagrange basis at the k+1 Gauss-Radau points)."""
import math
import os

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import timebasis as tb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "radau_iia.txt")


def _radau_iia():
    tabs, cur, k = {}, None, None
    s6 = math.sqrt(6.0)
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("k="):
            k = int(line[2:])
            tabs[k] = []
            continue
        tabs[k].append([eval(t, {"s6": s6}) for t in line.split(",")])
    return {k: np.array(v) for k, v in tabs.items()}


def test_radau_closed_forms():
    assert np.allclose(tb.radau_nodes(0), [1.0]) and np.allclose(tb.radau_weights(0), [1.0])
    assert np.allclose(tb.radau_nodes(1), [1 / 3, 1.0]) and np.allclose(tb.radau_weights(1), [0.75, 0.25])
    s6 = math.sqrt(6.0)
    assert np.allclose(tb.radau_nodes(2), [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-15)
    assert np.allclose(tb.radau_weights(2), [(16 - s6) / 36, (16 + s6) / 36, 1 / 9], atol=1e-15)


@pytest.mark.parametrize("k", range(5))
def test_radau_roots_and_exactness(k):
    c = tb.radau_nodes(k)
    w = tb.radau_weights(k)
    x = 2 * c - 1
    # roots of P_k - P_{k+1} (independent evaluation through scipy)
    assert np.max(np.abs(eval_legendre(k, x) - eval_legendre(k + 1, x))) < 1e-13
    assert c[-1] == 1.0 and np.all(np.diff(c) > 0) and c[0] > 0
    # exact for degree <= 2k, not for 2k+1; endpoint weight 1/(k+1)^2
    for q in range(2 * k + 1):
        assert abs(np.dot(w, c ** q) - 1.0 / (q + 1)) < 1e-14
    assert abs(np.dot(w, c ** (2 * k + 1)) - 1.0 / (2 * k + 2)) > 1e-6
    assert abs(w[-1] - 1.0 / (k + 1) ** 2) < 1e-14


def test_time_matrix_k1_closed_form():
    assert np.allclose(tb.time_matrix(1), [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]], atol=1e-15)
    assert np.allclose(tb.jump_vector(1), [1.5, -0.5], atol=1e-15)


@pytest.mark.parametrize("k", range(5))
def test_time_row_sums_equal_jump(k):
    # sum_b chi_b = 1, so sum_b T_ab = chi_a(0)
    assert np.allclose(tb.time_matrix(k).sum(axis=1), tb.jump_vector(k), atol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_dg_radau_equals_radau_iia(k):
    a = np.linalg.solve(tb.time_matrix(k), np.diag(tb.radau_weights(k)))
    assert np.allclose(a, _radau_iia()[k], atol=1e-13)


def _stability(k, z):
    """End value of the dG(k) slab for y' = lambda y, y(t_{n-1}) = 1, z = lambda tau."""
    m = tb.time_matrix(k) - z * np.diag(tb.radau_weights(k))
    return np.linalg.solve(m, tb.jump_vector(k))[-1]


@pytest.mark.parametrize("z", [-0.3, -2.0, 0.7, -10.0])
def test_stability_function_is_pade(z):
    # k = 0: implicit Euler 1/(1-z); k = 1: (k, k+1) Pade approximant of e^z
    assert abs(_stability(0, z) - 1.0 / (1.0 - z)) < 1e-14
    assert abs(_stability(1, z) - (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)) < 1e-13
    # k = 2: (2,3) Pade: (1 + 2z/5 + z^2/20) / (1 - 3z/5 + 3z^2/20 - z^3/60)
    assert abs(_stability(2, z) - (1 + 2 * z / 5 + z * z / 20) / (1 - 3 * z / 5 + 3 * z * z / 20 - z ** 3 / 60)) < 1e-13


@pytest.mark.parametrize("k", [2, 3, 4])
def test_time_matrix_against_high_precision(k):
    sp = pytest.importorskip("sympy")
    t, x = sp.symbols("t x")
    roots = sorted(sp.re(r) for r in sp.Poly(sp.legendre(k, x) - sp.legendre(k + 1, x), x).nroots(n=40))
    c = [(r + 1) / 2 for r in roots]
    chi = []
    for a in range(k + 1):
        pa = sp.Integer(1)
        for b in range(k + 1):
            if b != a:
                pa *= (t - c[b]) / (c[a] - c[b])
        chi.append(sp.expand(pa))
    ref = np.array([[float(sp.integrate(sp.diff(chi[b], t) * chi[a], (t, 0, 1)) + chi[a].subs(t, 0) * chi[b].subs(t, 0))
                     for b in range(k + 1)] for a in range(k + 1)])
    wref = np.array([float(sp.integrate(ch, (t, 0, 1))) for ch in chi])
    assert np.abs(tb.time_matrix(k) - ref).max() < 1e-14 * np.abs(ref).max()
    assert np.abs(tb.radau_weights(k) - wref).max() < 1e-15
