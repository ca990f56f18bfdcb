"""Pins of the oracle's element, assembly and right-hand side (Sec. 2, Eq. (2.1)-(2.2), Eq. (3.3)).

The strongest pin is Galerkin exactness: a velocity that is quadratic in space
and linear in time, with a pressure linear in space and time, lies in the
discrete space; Nitsche's method is consistent and every integral below is
exact for these degrees, so its interpolant solves the discrete slab problem
to rounding.  A missing or mis-signed term of A_h, of B_GammaD, of the time
derivative, of the jump or of the right-hand side breaks that identity.
"""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, element, mesh, multigrid, timebasis

NU = 0.05
TAU = 0.3
T0 = 0.2


# --- manufactured solution: div-free quadratic velocity, linear pressure ------------------------
def vel(x, t):
    if x.shape[1] == 2:
        X, Y = x[:, 0], x[:, 1]
        return np.stack([X * X + t * Y * Y, -2 * X * Y + t * X * X], 1)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return np.stack([X * X + t * Y * Y, -2 * X * Y + t * Z * Z, t * X * X + 0 * Z], 1)


def vel_t(x):
    if x.shape[1] == 2:
        return np.stack([x[:, 1] ** 2, x[:, 0] ** 2], 1)
    return np.stack([x[:, 1] ** 2, x[:, 2] ** 2, x[:, 0] ** 2], 1)


def vel_grad(x, t):
    """G[:, c, e] = d v_c / d x_e."""
    n, d = x.shape
    g = np.zeros((n, d, d))
    X, Y = x[:, 0], x[:, 1]
    g[:, 0, 0] = 2 * X
    g[:, 0, 1] = 2 * t * Y
    g[:, 1, 0] = -2 * Y + (2 * t * X if d == 2 else 0)
    g[:, 1, 1] = -2 * X
    if d == 3:
        Z = x[:, 2]
        g[:, 1, 2] = 2 * t * Z
        g[:, 2, 0] = 2 * t * X
    return g


def vel_lap(x, t):
    d = x.shape[1]
    if d == 2:
        return np.stack([2 + 2 * t + 0 * x[:, 0], 0 * x[:, 0] + 2 * t], 1)
    return np.stack([2 + 2 * t + 0 * x[:, 0], 0 * x[:, 0] + 2 * t, 0 * x[:, 0] + 2 * t], 1)


def pres(x, t):
    return x[:, 0] + 2 * x[:, 1] - 0.7 + t * (x[:, 0] - x[:, 1])


def pres_grad(x, t):
    g = np.zeros_like(x)
    g[:, 0] = 1 + t
    g[:, 1] = 2 - t
    return g


def wfield(x):
    """Linearisation velocity, in Q2 (so its nodal interpolant is exact)."""
    if x.shape[1] == 2:
        return np.stack([0.5 + x[:, 0] * x[:, 1], x[:, 0] ** 2 - 0.3 * x[:, 1]], 1)
    return np.stack([0.5 + x[:, 0] * x[:, 1], x[:, 0] ** 2 - 0.3 * x[:, 2], x[:, 1] * x[:, 2]], 1)


def forcing(nu):
    def f(x, t):
        w = wfield(x)
        conv = np.einsum("ne,nce->nc", w, vel_grad(x, t))
        return vel_t(x) + conv - nu * vel_lap(x, t) + pres_grad(x, t)
    return f


def interpolant(lev, t0, tau):
    k, d = lev.k, lev.dim
    cn = timebasis.radau_nodes(k)
    xn = lev.node_coords()
    cen = lev.cell_centres()
    h = np.asarray(lev.h)
    x = np.zeros(lev.N)
    for a in range(k + 1):
        ta = t0 + tau * cn[a]
        x[lev.vel_index(a, np.arange(lev.n_nodes)[:, None], np.arange(d)[None, :])] = vel(xn, ta)
        x[lev.pres_index(a, np.arange(lev.n_cells), 0)] = pres(cen, ta)
        g = pres_grad(cen, ta)
        for e in range(d):
            x[lev.pres_index(a, np.arange(lev.n_cells), e + 1)] = g[:, e] * h[e] / 2
    return x


def traction_rhs(lev, nu, t0, tau):
    """tau w_a <(nu grad v - p I) n, psi_i> on the do-nothing faces (not part of the discrete RHS)."""
    k, d = lev.k, lev.dim
    h = np.asarray(lev.h)
    cn = timebasis.radau_nodes(k)
    wts = timebasis.radau_weights(k)
    out = np.zeros(lev.N)
    cen = lev.cell_centres()
    for e, side, cells in lev.boundary_faces():
        if lev.is_dirichlet(e, side):
            continue
        fp, fw = element.face_rule(d, e, side)
        fqw = fw * np.prod(np.delete(h, e) / 2)
        fv, _ = element.q2_basis(fp)
        nrm = np.zeros(d)
        nrm[e] = 1.0 if side else -1.0
        xf = (cen[cells][:, None, :] + fp[None] * (h / 2)).reshape(-1, d)
        for a in range(k + 1):
            ta = t0 + tau * cn[a]
            tr = nu * vel_grad(xf, ta) @ nrm - pres(xf, ta)[:, None] * nrm[None, :]
            tr = tr.reshape(len(cells), -1, d)
            loc = tau * wts[a] * np.einsum("q,qi,kqc->kic", fqw, fv, tr)
            idx = lev.vel_index(a, lev.cell_nodes[cells][:, :, None], np.arange(d)[None, None, :])
            np.add.at(out, idx, loc)
    return out


def nodal_w(lev):
    wn = wfield(lev.node_coords())
    return np.repeat(wn.reshape(1, -1), lev.k + 1, axis=0)


def manufactured_residual(spec, k):
    lev = mesh.Level(spec, spec.n_levels - 1, k)
    jac = assemble.jacobian(lev, nodal_w(lev), NU, TAU, newton=False)
    x = interpolant(lev, T0, TAU)
    vprev = vel(lev.node_coords(), T0).ravel()
    b = assemble.rhs_linear(lev, forcing(NU), lambda xx, t: vel(xx, t), vprev, NU, TAU, T0)
    b = b + traction_rhs(lev, NU, T0, TAU)
    return np.linalg.norm(jac @ x - b) / np.linalg.norm(b)


SPECS = {
    "square_dirichlet": si.MeshSpec(2, (3, 2), (0.0, 0.0), (1.0, 0.7), 1, si.ALL2),
    "square_outflow": si.MeshSpec(2, (3, 2), (0.1, 0.0), (1.3, 0.7), 1,
                                  si.FACE_XLO | si.FACE_YLO | si.FACE_YHI),
    "cube_dirichlet": si.MeshSpec(3, (2, 1, 2), (0.0,) * 3, (1.0, 0.5, 0.8), 1, si.ALL3),
    "cube_outflow": si.MeshSpec(3, (2, 1, 2), (0.0,) * 3, (1.0, 0.5, 0.8), 1, si.ALL3 & ~si.FACE_XHI),
}


# 2D at k = 0, 1, 2; 3D at k = 0, 1 (k = 2 in 3D adds run time and no new term)
@pytest.mark.parametrize("name,k", [(n, k) for n in SPECS for k in (0, 1, 2) if not (n.startswith("cube") and k == 2)])
def test_galerkin_exactness(name, k):
    assert manufactured_residual(SPECS[name], k) < 1e-12


def test_q2_basis_and_rules():
    pts = np.random.default_rng(0).uniform(-1, 1, (7, 2))
    v, g = element.q2_basis(pts)
    assert np.allclose(v.sum(1), 1) and np.allclose(g.sum(1), 0)
    nodes = element.local_nodes(2) - 1.0
    vn, _ = element.q2_basis(nodes)
    assert np.allclose(vn, np.eye(9))
    p, w = element.cell_rule(2)
    for q in range(6):
        assert abs(np.dot(w, p[:, 0] ** q) - (2 / (q + 1) if q % 2 == 0 else 0) * 2) < 1e-14
    assert abs(np.dot(w, p[:, 0] ** 6) - 2 / 7 * 2) > 1e-4


def test_mass_and_stiffness_invariants():
    lev = mesh.Level(SPECS["square_dirichlet"], 0, 0)
    m = assemble.mass_matrix(lev)
    assert abs(m.sum() - 2 * 0.7) < 1e-13          # d * |Omega|
    ops = assemble.CellOperators(lev, np.zeros((1, lev.R)), NU, False)
    assert np.allclose(ops.stiff.sum(1), 0, atol=1e-13)


def _blocks(lev, jac, a, b):
    ra = slice(a * (lev.R + lev.S), a * (lev.R + lev.S) + lev.R)
    pa = slice(a * (lev.R + lev.S) + lev.R, (a + 1) * (lev.R + lev.S))
    rb = slice(b * (lev.R + lev.S), b * (lev.R + lev.S) + lev.R)
    pb = slice(b * (lev.R + lev.S) + lev.R, (b + 1) * (lev.R + lev.S))
    j = jac.toarray()
    return j[ra, rb], j[ra, pb], j[pa, rb], j[pa, pb]


@pytest.mark.parametrize("name", ["square_dirichlet", "cube_outflow"])
def test_symmetric_nitsche_without_convection(name):
    lev = mesh.Level(SPECS[name], 0, 0)
    jac = assemble.jacobian(lev, np.zeros((1, lev.R)), NU, TAU, newton=False)
    vv, vp, pv, pp = _blocks(lev, jac, 0, 0)
    assert np.allclose(vv, vv.T, atol=1e-14)
    assert np.allclose(vp, -pv.T, atol=1e-14)
    assert np.all(pp == 0)


@pytest.mark.parametrize("k", [1, 2])
def test_time_structure(k):
    lev = mesh.Level(SPECS["square_outflow"], 0, k)
    jac = assemble.jacobian(lev, nodal_w(lev), NU, TAU, newton=True)
    m = assemble.mass_matrix(lev).toarray()
    tm = timebasis.time_matrix(k)
    for a in range(k + 1):
        for b in range(k + 1):
            vv, vp, pv, pp = _blocks(lev, jac, a, b)
            if a != b:
                assert np.allclose(vv, tm[a, b] * m, atol=1e-14)
                assert np.all(vp == 0) and np.all(pv == 0)
            else:
                assert np.allclose(vp, -pv.T, atol=1e-14)


@pytest.mark.parametrize("spec", [SPECS["square_dirichlet"], SPECS["cube_dirichlet"]])
def test_constant_pressure_null_vectors(spec):
    k = 1
    lev = mesh.Level(spec, 0, k)
    jac = assemble.jacobian(lev, nodal_w(lev), NU, TAU, newton=True)
    for a in range(k + 1):
        e = np.zeros(lev.N)
        e[lev.pres_index(a, np.arange(lev.n_cells), 0)] = 1.0
        assert np.linalg.norm(jac @ e) < 1e-13
        assert np.linalg.norm(jac.T @ e) < 1e-13
    c = multigrid.pressure_mean_vectors(lev)
    assert c.shape == (k + 1, lev.N)


@pytest.mark.parametrize("name", ["square_outflow", "cube_dirichlet"])
def test_newton_term_is_convection_derivative(name):
    # d/dv ((v.grad)v, psi) [delta] at w = ((w.grad)delta, psi) + ((delta.grad)w, psi):
    # (J_newton(w) - J_oseen(w)) delta == (J_oseen(delta) - J_oseen(0)) w
    lev = mesh.Level(SPECS[name], 0, 1)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((2, lev.R))
    dl = rng.standard_normal((2, lev.R))

    def full(v):
        x = np.zeros(lev.N)
        for a in range(2):
            x[a * (lev.R + lev.S):a * (lev.R + lev.S) + lev.R] = v[a]
        return x

    jn = assemble.jacobian(lev, w, NU, TAU, True)
    jo = assemble.jacobian(lev, w, NU, TAU, False)
    jd = assemble.jacobian(lev, dl, NU, TAU, False)
    j0 = assemble.jacobian(lev, np.zeros_like(dl), NU, TAU, False)
    lhs = (jn - jo) @ full(dl)
    rhs = (jd - j0) @ full(w)
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(rhs)


# --- planted mistakes: each must break one of the pins above ----------------------------------
def test_planted_mistakes_are_caught(monkeypatch):
    spec = SPECS["square_outflow"]
    assert manufactured_residual(spec, 1) < 1e-12
    jump, tmat, wts = timebasis.jump_vector, timebasis.time_matrix, timebasis.radau_weights
    mistakes = {
        "jump dropped": ("jump_vector", lambda k: 0 * jump(k)),
        "time matrix transposed": ("time_matrix", lambda k: tmat(k).T),
        "weights reversed": ("radau_weights", lambda k: wts(k)[::-1]),
    }
    for label, (name, repl) in mistakes.items():
        monkeypatch.setattr(timebasis, name, repl)
        assert manufactured_residual(spec, 1) > 1e-6, label
        monkeypatch.undo()
    # B_GammaD's penalty enters J and the right-hand side alike, so exactness cannot see its
    # sign; coercivity does: with gamma2 < 0 the Stokes-Nitsche velocity block is indefinite.
    lev = mesh.Level(si.MeshSpec(2, (2, 2), (0, 0), (1, 1), 1, si.ALL2), 0, 0)
    jac = assemble.jacobian(lev, np.zeros((1, lev.R)), NU, TAU, False, gamma2=-35.0)
    assert np.min(np.linalg.eigvalsh(jac.toarray()[:lev.R, :lev.R])) < 0


def test_penalty_makes_velocity_block_definite():
    lev = mesh.Level(si.MeshSpec(2, (2, 2), (0, 0), (1, 1), 1, si.ALL2), 0, 0)
    jac = assemble.jacobian(lev, np.zeros((1, lev.R)), NU, TAU, False)
    vv = jac.toarray()[:lev.R, :lev.R]
    assert np.min(np.linalg.eigvalsh(vv)) > 0
