"""Pins of the oracle's (Q4)^2 x P3disc element (the pair of the paper's 2D experiment, Sec. 2:
(Q_r)^d x P_{r-1}^disc with r = 4).

* The element: Q4 Lagrange functions are a partition of unity with the Kronecker property at the
  equidistant nodes; the 5-point Gauss rule integrates degree 9 exactly and not degree 10; the P3
  monomials number 10.
* Galerkin exactness: a divergence-free velocity of degree 4 in space (the curl of a degree-5
  stream function) and linear in time, with a cubic pressure, lies in the discrete space; Nitsche's
  method is consistent and the viscous, pressure, mass and face integrals are exact for these
  degrees with the 5-point rule (the convection uses the same rule on both sides), so its
  interpolant solves the discrete slab problem to rounding (k = 0, 1, 2; all-Dirichlet box and a
  do-nothing face; Oseen and Newton).
* Transfers: the prolongation reproduces coarse Q4 and P3 functions at arbitrary points.
* Smoother and solver: the one-cell Vanka closed form, the dense averaged-sweep formula, and
  FGMRES with the V-cycle against a dense solve.
"""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, element, fgmres, mesh, multigrid, timebasis, transfer, vanka

NU, TAU, T0 = 0.05, 0.3, 0.2
R4 = 4
OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI


def _psi_grad(x, c):
    """Gradient of psi = c0 x^3 y^2 + c1 x y^4 + c2 x^5 + c3 y^5 + c4 x^2 y^3."""
    X, Y = x[:, 0], x[:, 1]
    px = 3 * c[0] * X**2 * Y**2 + c[1] * Y**4 + 5 * c[2] * X**4 + 2 * c[4] * X * Y**3
    py = 2 * c[0] * X**3 * Y + 4 * c[1] * X * Y**3 + 5 * c[3] * Y**4 + 3 * c[4] * X**2 * Y**2
    return px, py


C0, C1 = (0.3, -0.2, 0.1, 0.15, -0.25), (-0.1, 0.2, 0.05, -0.3, 0.1)


def vel(x, t):
    px0, py0 = _psi_grad(x, C0)
    px1, py1 = _psi_grad(x, C1)
    return np.stack([py0 + t * py1, -px0 - t * px1], 1)


def vel_t(x):
    px1, py1 = _psi_grad(x, C1)
    return np.stack([py1, -px1], 1)


def vel_grad(x, t, h=1e-5):
    """d v_c / d x_e by central differences of the polynomial (exact to ~1e-10 relative)."""
    g = np.zeros((len(x), 2, 2))
    for e in range(2):
        dx = np.zeros(2)
        dx[e] = h
        g[:, :, e] = (vel(x + dx, t) - vel(x - dx, t)) / (2 * h)
    return g


def _psi_hess_derivs(x, c):
    """Laplacian of (psi_y, -psi_x) for the quintic psi, analytically."""
    X, Y = x[:, 0], x[:, 1]
    # psi_y = 2c0 x^3 y + 4c1 x y^3 + 5c3 y^4 + 3c4 x^2 y^2
    lap_py = (12 * c[0] * X * Y + 24 * c[1] * X * Y + 60 * c[3] * Y**2 + 6 * c[4] * Y**2 + 6 * c[4] * X**2)
    # psi_x = 3c0 x^2 y^2 + c1 y^4 + 5c2 x^4 + 2c4 x y^3
    lap_px = (6 * c[0] * Y**2 + 6 * c[0] * X**2 + 12 * c[1] * Y**2 + 60 * c[2] * X**2 + 12 * c[4] * X * Y)
    return np.stack([lap_py, -lap_px], 1)


def vel_lap(x, t):
    return _psi_hess_derivs(x, C0) + t * _psi_hess_derivs(x, C1)


def pres(x, t):
    X, Y = x[:, 0], x[:, 1]
    return X**3 - 0.5 * X * Y**2 + 0.3 * Y**3 - 0.2 + t * (X**2 * Y - Y)


def pres_grad(x, t):
    X, Y = x[:, 0], x[:, 1]
    return np.stack([3 * X**2 - 0.5 * Y**2 + t * 2 * X * Y, -X * Y + 0.9 * Y**2 + t * (X**2 - 1)], 1)


def wfield(x):
    """Linearisation velocity in Q4 (its nodal interpolant is exact)."""
    return np.stack([0.5 + x[:, 0] ** 2 * x[:, 1], x[:, 0] * x[:, 1] ** 3 - 0.3 * x[:, 1]], 1)


def nodal_w(lev):
    return np.repeat(wfield(lev.node_coords()).reshape(1, -1), lev.k + 1, axis=0)


def pres_coefficients(lev, t):
    """P3disc coefficients of the cubic pressure on every cell (exact solve at the Gauss points)."""
    pts, _ = element.cell_rule_r(2, R4)
    B = element.pdisc_basis(R4, pts)
    cen, h = lev.cell_centres(), np.asarray(lev.h)
    out = np.zeros((lev.n_cells, lev.Shat))
    for c in range(lev.n_cells):
        vals = pres(cen[c] + pts * h / 2, t)
        out[c] = np.linalg.lstsq(B, vals, rcond=None)[0]
    return out


def interpolant(lev, t0, tau):
    cn = timebasis.radau_nodes(lev.k)
    xn = lev.node_coords()
    x = np.zeros(lev.N)
    for a in range(lev.k + 1):
        ta = t0 + tau * cn[a]
        x[lev.vel_index(a, np.arange(lev.n_nodes)[:, None], np.arange(2)[None, :])] = vel(xn, ta)
        x[lev.pres_index(a, np.arange(lev.n_cells)[:, None], np.arange(lev.Shat)[None, :])] = pres_coefficients(lev, ta)
    return x


def traction_rhs(lev, nu, t0, tau):
    k, h = lev.k, np.asarray(lev.h)
    cn, wts = timebasis.radau_nodes(k), timebasis.radau_weights(k)
    out = np.zeros(lev.N)
    cen = lev.cell_centres()
    for e, side, cells in lev.boundary_faces():
        if lev.is_dirichlet(e, side):
            continue
        fp, fw = element.face_rule_r(2, e, side, R4)
        fqw = fw * np.prod(np.delete(h, e) / 2)
        fv, _ = element.q_basis(R4, fp)
        nrm = np.zeros(2)
        nrm[e] = 1.0 if side else -1.0
        xf = (cen[cells][:, None, :] + fp[None] * (h / 2)).reshape(-1, 2)
        for a in range(k + 1):
            ta = t0 + tau * cn[a]
            tr = nu * vel_grad(xf, ta) @ nrm - pres(xf, ta)[:, None] * nrm[None, :]
            tr = tr.reshape(len(cells), -1, 2)
            loc = tau * wts[a] * np.einsum("q,qi,kqc->kic", fqw, fv, tr)
            idx = lev.vel_index(a, lev.cell_nodes[cells][:, :, None], np.arange(2)[None, None, :])
            np.add.at(out, idx, loc)
    return out


def residual(spec, k, newton=False):
    lev = mesh.Level(spec, spec.n_levels - 1, k)
    jac = assemble.jacobian(lev, nodal_w(lev), NU, TAU, newton=False)

    def f(x, t):
        conv = np.einsum("ne,nce->nc", wfield(x), vel_grad(x, t))
        return vel_t(x) + conv - NU * vel_lap(x, t) + pres_grad(x, t)
    b = assemble.rhs_linear(lev, f, lambda xx, t: vel(xx, t), vel(lev.node_coords(), T0).ravel(), NU, TAU, T0)
    b = b + traction_rhs(lev, NU, T0, TAU)
    x = interpolant(lev, T0, TAU)
    return np.linalg.norm(jac @ x - b) / np.linalg.norm(b)


SPECS = {
    "box_dirichlet": si.MeshSpec(2, (2, 2), (0.0, 0.0), (1.0, 0.7), 1, si.ALL2, order=4),
    "box_outflow": si.MeshSpec(2, (3, 2), (0.1, 0.0), (1.3, 0.7), 1, OUT2, order=4),
}


def test_q4_element_and_rules():
    nodes = -1.0 + 2.0 * element.local_nodes_r(2, 4) / 4
    v, g = element.q_basis(4, nodes)
    assert np.allclose(v, np.eye(25), atol=1e-13)
    pts = np.random.default_rng(0).uniform(-1, 1, (9, 2))
    v, g = element.q_basis(4, pts)
    assert np.allclose(v.sum(1), 1) and np.allclose(g.sum(1), 0, atol=1e-12)
    x, w = element.gauss_rule_1d(4)
    for q in range(10):
        assert abs(np.dot(w, x ** q) - (2 / (q + 1) if q % 2 == 0 else 0)) < 1e-14
    assert abs(np.dot(w, x ** 10) - 2 / 11) > 1e-6
    xl, wl = np.polynomial.legendre.leggauss(5)            # the closed form is the Gauss-Legendre rule
    assert np.allclose(x, xl, rtol=0, atol=1e-15) and np.allclose(w, wl, rtol=0, atol=1e-15)
    assert len(element.pdisc_exponents(4, 2)) == 10
    lev = mesh.Level(SPECS["box_dirichlet"], 0, 1)
    assert (lev.n_patch, lev.nn) == (60 * 2, (9, 9))


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("k", [0, 1, 2])
def test_q4_galerkin_exactness(name, k):
    assert residual(SPECS[name], k) < 1e-11


def _fe_eval(lev, x, pts):
    u = (pts - np.asarray(lev.spec.lo)) / np.asarray(lev.h)
    ci = np.clip(np.floor(u).astype(int), 0, np.asarray(lev.cells) - 1)
    ref = 2 * (u - ci) - 1
    cell = ci[:, 0] + lev.cells[0] * ci[:, 1]
    vals, _ = element.q_basis(lev.r, ref)
    v = np.einsum("pi,pic->pc", vals, x[:lev.R].reshape(-1, 2)[lev.cell_nodes[cell]])
    pc = x[lev.R:lev.R + lev.S].reshape(-1, lev.Shat)[cell]
    p = np.einsum("pm,pm->p", element.pdisc_basis(lev.r, ref), pc)
    return v, p


def test_q4_prolongation_reproduces_coarse_functions():
    spec = si.MeshSpec(2, (4, 2), (0.0, 0.0), (1.0, 0.6), 2, si.ALL2, order=4)
    coarse, fine = mesh.Level(spec, 0, 0), mesh.Level(spec, 1, 0)
    P = transfer.prolongation(coarse, fine)
    xc = np.random.default_rng(1).standard_normal(coarse.N)
    xf = P @ xc
    pts = np.random.default_rng(2).uniform(0.001, 0.999, (200, 2)) * np.asarray(spec.hi)
    vc, pc = _fe_eval(coarse, xc, pts)
    vf, pf = _fe_eval(fine, xf, pts)
    assert np.allclose(vc, vf, atol=1e-12) and np.allclose(pc, pf, atol=1e-12)


def test_q4_one_cell_vanka_and_dense_sweep():
    spec = si.MeshSpec(2, (1, 1), (0.0, 0.0), (1.0, 1.0), 1, OUT2, order=4)
    lev = mesh.Level(spec, 0, 1)
    w = np.random.default_rng(5).uniform(-1, 1, (2, lev.R))
    jac = assemble.jacobian(lev, w, NU, TAU, True)
    b = np.random.default_rng(0).standard_normal(lev.N)
    xs = np.linalg.solve(jac.toarray(), b)
    d = vanka.sweep_averaged(jac, lev, vanka.local_inverses(jac, lev), b, np.zeros(lev.N), 0.7, 2)
    assert np.allclose(d, (1 - 0.3 ** 2) * xs, rtol=1e-10, atol=1e-11)
    spec = si.MeshSpec(2, (2, 2), (0.0, 0.0), (1.0, 1.0), 1, OUT2, order=4)
    lev = mesh.Level(spec, 0, 0)
    w = np.random.default_rng(5).uniform(-1, 1, (1, lev.R))
    jac = assemble.jacobian(lev, w, NU, TAU, True)
    jd = jac.toarray()
    ext = []
    for cell in range(lev.n_cells):
        m = np.zeros((lev.N, lev.n_patch))
        m[lev.dof[cell], np.arange(lev.n_patch)] = 1.0
        ext.append(m)
    count = sum(e @ np.ones(lev.n_patch) for e in ext)
    b = np.random.default_rng(1).standard_normal(lev.N)
    d_ref = np.random.default_rng(2).standard_normal(lev.N)
    d = vanka.sweep_averaged(jac, lev, vanka.local_inverses(jac, lev), b, d_ref, 0.7, 2)
    for _ in range(2):
        corr = sum(e @ np.linalg.solve(e.T @ jd @ e, e.T @ (b - jd @ d_ref)) for e in ext)
        d_ref = d_ref + 0.7 * corr / count
    assert np.allclose(d, d_ref, rtol=1e-10, atol=1e-11)


def test_q4_fgmres_matches_dense_solve():
    spec = si.MeshSpec(2, (4, 2), (0.0, 0.0), (2.2, 0.41), 2, OUT2, order=4)
    w = si.channel_w(spec, 1)
    h = multigrid.Hierarchy(spec, 1, 1e-3, 0.01, w, newton=True, nu1=2, nu2=2)
    b = h.apply(si.reference_solution(spec, 1))
    x, its, rel, ok = fgmres.fgmres(h.apply, h.vcycle, b, rtol=1e-12)
    xd = np.linalg.solve(h.J[-1].toarray(), b)
    assert ok and np.linalg.norm(x - xd) < 1e-9 * np.linalg.norm(xd)
    assert its <= 30


def test_q4_exactness_catches_planted_mistakes(monkeypatch):
    """Galerkin exactness fails for two plausible mistakes: Lagrange functions built on other nodes
    (Gauss-Lobatto instead of equidistant) than the nodes the unknowns sit at, and a pressure
    space of degree 2 instead of 3."""
    spec = SPECS["box_outflow"]
    assert residual(spec, 1) < 1e-11
    s37 = np.sqrt(3.0 / 7.0)
    lob = np.array([-1.0, -s37, 0.0, s37, 1.0])
    orig = element.lagrange1d_r

    def lagrange_on_lobatto(r, x):
        x = np.asarray(x, float)
        if r != 4:
            return orig(r, x)
        vals = np.ones(x.shape + (5,))
        ders = np.zeros(x.shape + (5,))
        for l in range(5):
            others = [m for m in range(5) if m != l]
            den = np.prod([lob[l] - lob[m] for m in others])
            for m in others:
                vals[..., l] *= x - lob[m]
            for q in others:
                term = np.ones(x.shape)
                for m in others:
                    if m != q:
                        term = term * (x - lob[m])
                ders[..., l] += term
            vals[..., l] /= den
            ders[..., l] /= den
        return vals, ders
    monkeypatch.setattr(element, "lagrange1d_r", lagrange_on_lobatto)
    assert residual(spec, 1) > 1e-6
    monkeypatch.undo()
    exps = element.pdisc_exponents
    monkeypatch.setattr(element, "pdisc_exponents", lambda r, d: [a for a in exps(r, d) if sum(a) <= 2])
    assert residual(spec, 1) > 1e-6
