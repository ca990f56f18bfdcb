"""Pins of the oracle's transfers, Vanka smoother (Eq. (3.4), (S0)-(S3)), V-cycle and FGMRES (Sec. 3).

The smoother is checked against the closed form on a one-cell mesh and against
dense brute force built from explicit extension matrices E_K and numpy's
inverse of every J_K; the V-cycle against an independent dense operator; the
FGMRES solution against a dense direct solve.
"""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, element, fgmres, mesh, multigrid, transfer, vanka

NU, TAU = 1e-2, 0.05
OUTFLOW2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI


def _w(lev, seed=5):
    return np.random.default_rng(seed).uniform(-1, 1, (lev.k + 1, lev.R))


def _fe_eval(lev, x, pts):
    """Evaluate the FE velocity/pressure of coefficient vector x (time node 0) at points."""
    d = lev.dim
    u = (pts - np.asarray(lev.spec.lo)) / np.asarray(lev.h)
    ci = np.clip(np.floor(u).astype(int), 0, np.asarray(lev.cells) - 1)
    ref = 2 * (u - ci) - 1
    cell = sum(ci[:, e] * int(np.prod(lev.cells[:e])) for e in range(d))
    vals, _ = element.q2_basis(ref)
    vel = x[:lev.R].reshape(-1, d)[lev.cell_nodes[cell]]          # (npts, nloc, d)
    v = np.einsum("pi,pic->pc", vals, vel)
    pc = x[lev.R:lev.R + lev.S].reshape(-1, d + 1)[cell]
    p = np.einsum("pm,pm->p", element.p1disc_basis(ref), pc)
    return v, p


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_reproduces_coarse_functions(dim):
    spec = si.MeshSpec(dim, (4,) * dim, (0.0,) * dim, (1.0, 0.6, 0.8)[:dim], 2, (1 << 2 * dim) - 1)
    coarse, fine = mesh.Level(spec, 0, 0), mesh.Level(spec, 1, 0)
    p = transfer.prolongation(coarse, fine)
    xc = np.random.default_rng(1).standard_normal(coarse.N)
    xf = p @ xc
    pts = np.random.default_rng(2).uniform(0.001, 0.999, (200, dim)) * np.asarray(spec.hi)
    vc, pc = _fe_eval(coarse, xc, pts)
    vf, pf = _fe_eval(fine, xf, pts)
    assert np.allclose(vc, vf, atol=1e-13) and np.allclose(pc, pf, atol=1e-13)


def test_prolongation_1d_weights():
    spec = si.MeshSpec(2, (2, 2), (0.0, 0.0), (1.0, 1.0), 2, si.ALL2)
    coarse, fine = mesh.Level(spec, 0, 0), mesh.Level(spec, 1, 0)
    p = transfer.prolongation(coarse, fine).toarray()
    # fine node (1, 0) lies at xi = -1/2 of coarse cell 0 on the edge y = 0: weights 3/8, 3/4, -1/8
    row = p[fine.vel_index(0, 1, 0)]
    cols = [coarse.vel_index(0, n, 0) for n in range(3)]
    assert np.allclose(row[cols], [3 / 8, 3 / 4, -1 / 8], atol=1e-15)
    assert np.isclose(row.sum(), 1.0)


def test_one_cell_vanka_is_damped_exact_solve():
    spec = si.MeshSpec(2, (1, 1), (0.0, 0.0), (1.0, 1.0), 1, OUTFLOW2)
    for k in (0, 1):
        lev = mesh.Level(spec, 0, k)
        jac = assemble.jacobian(lev, _w(lev), NU, TAU, True)
        jinv = vanka.local_inverses(jac, lev)
        b = np.random.default_rng(0).standard_normal(lev.N)
        xs = np.linalg.solve(jac.toarray(), b)
        for j in (1, 2, 3):
            d = vanka.sweep_averaged(jac, lev, jinv, b, np.zeros(lev.N), 0.7, j)
            assert np.allclose(d, (1 - 0.3 ** j) * xs, rtol=1e-11, atol=1e-12)


def _extensions(lev):
    e = []
    for cell in range(lev.n_cells):
        m = np.zeros((lev.N, lev.n_patch))
        m[lev.dof[cell], np.arange(lev.n_patch)] = 1.0
        e.append(m)
    return e


@pytest.mark.parametrize("cells,k", [((2, 2), 0), ((3, 2), 1), ((4, 4), 0)])
def test_averaged_sweep_matches_dense_formula(cells, k):
    spec = si.MeshSpec(2, cells, (0.0, 0.0), (1.0, 1.0), 1, OUTFLOW2)
    lev = mesh.Level(spec, 0, k)
    jac = assemble.jacobian(lev, _w(lev), NU, TAU, True)
    jd = jac.toarray()
    ext = _extensions(lev)
    blocks = [np.linalg.inv(e.T @ jd @ e) for e in ext]
    count = sum(e @ np.ones(lev.n_patch) for e in ext)
    b = np.random.default_rng(1).standard_normal(lev.N)
    d_ref = np.random.default_rng(2).standard_normal(lev.N)
    d = vanka.sweep_averaged(jac, lev, vanka.local_inverses(jac, lev), b, d_ref, 0.7, 3)
    for _ in range(3):
        corr = sum(e @ bk @ e.T @ (b - jd @ d_ref) for e, bk in zip(ext, blocks))
        d_ref = d_ref + 0.7 * corr / count
    assert np.allclose(d, d_ref, rtol=1e-11, atol=1e-12)


def test_coloured_sweep_matches_dense_formula():
    spec = si.MeshSpec(2, (4, 3), (0.0, 0.0), (1.0, 1.0), 1, OUTFLOW2)
    lev = mesh.Level(spec, 0, 1)
    jac = assemble.jacobian(lev, _w(lev), NU, TAU, True)
    jd = jac.toarray()
    ext = _extensions(lev)
    b = np.random.default_rng(1).standard_normal(lev.N)
    d_ref = np.zeros(lev.N)
    d = vanka.sweep_coloured(jac, lev, vanka.local_inverses(jac, lev), b, d_ref, 0.7, 2)
    for _ in range(2):
        for colour in range(4):
            r = b - jd @ d_ref
            for cell in np.nonzero(lev.colour == colour)[0]:
                e = ext[cell]
                d_ref = d_ref + 0.7 * e @ np.linalg.solve(e.T @ jd @ e, e.T @ r)
    assert np.allclose(d, d_ref, rtol=1e-11, atol=1e-12)


def test_colours_share_no_velocity_dof():
    for dim, cells in ((2, (5, 4)), (3, (3, 4, 2))):
        lev = mesh.Level(si.MeshSpec(dim, cells, (0.0,) * dim, (1.0,) * dim, 1, 0), 0, 1)
        for colour in range(2 ** dim):
            nodes = lev.cell_nodes[lev.colour == colour].ravel()
            assert len(nodes) == len(np.unique(nodes))


def _hier(spec, k, nu1=2, nu2=2, smoother="averaged"):
    lev = mesh.Level(spec, spec.n_levels - 1, k)
    return multigrid.Hierarchy(spec, k, NU, TAU, _w(lev), newton=True, nu1=nu1, nu2=nu2, smoother=smoother)


def test_single_level_cycle_is_direct_solve():
    spec = si.MeshSpec(2, (3, 2), (0.0, 0.0), (1.0, 1.0), 1, OUTFLOW2)
    h = _hier(spec, 1)
    b = np.random.default_rng(0).standard_normal(h.fine.N)
    assert np.allclose(h.J[0] @ h.vcycle(b), b, atol=1e-11)


def test_singular_coarse_solve_is_zero_mean_solution():
    spec = si.MeshSpec(2, (3, 2), (0.0, 0.0), (1.0, 1.0), 1, si.ALL2)
    h = _hier(spec, 1)
    xs = si.reference_solution(spec, 1)
    b = h.J[0] @ xs
    x = h.vcycle(b)
    assert np.allclose(x, xs, atol=1e-9)


@pytest.mark.parametrize("smoother", ["averaged", "coloured"])
def test_two_level_cycle_matches_dense_operator(smoother):
    spec = si.MeshSpec(2, (4, 4), (0.0, 0.0), (1.0, 1.0), 2, OUTFLOW2)
    h = _hier(spec, 1, nu1=2, nu2=1, smoother=smoother)
    fine = h.fine
    jf, jc = h.J[1].toarray(), h.J[0].toarray()
    p = h.P[1].toarray()
    ext = _extensions(fine)
    count = sum(e @ np.ones(fine.n_patch) for e in ext)

    def smooth(d, b, n):
        for _ in range(n):
            if smoother == "averaged":
                r = b - jf @ d
                d = d + 0.7 * sum(e @ np.linalg.solve(e.T @ jf @ e, e.T @ r) for e in ext) / count
            else:
                for colour in range(4):
                    r = b - jf @ d
                    for cell in np.nonzero(fine.colour == colour)[0]:
                        e = ext[cell]
                        d = d + 0.7 * e @ np.linalg.solve(e.T @ jf @ e, e.T @ r)
        return d

    b = np.random.default_rng(4).standard_normal(fine.N)
    d = smooth(np.zeros(fine.N), b, 2)
    d = d + p @ np.linalg.solve(jc, p.T @ (b - jf @ d))
    d = smooth(d, b, 1)
    assert np.allclose(h.vcycle(b), d, rtol=1e-10, atol=1e-11)


def test_vcycle_is_linear():
    spec = si.MeshSpec(2, (4, 4), (0.0, 0.0), (1.0, 1.0), 2, OUTFLOW2)
    h = _hier(spec, 0)
    rng = np.random.default_rng(3)
    b1, b2 = rng.standard_normal((2, h.fine.N))
    assert np.allclose(h.vcycle(2 * b1 - 3 * b2), 2 * h.vcycle(b1) - 3 * h.vcycle(b2), atol=1e-10)


def test_fgmres_small_dense():
    rng = np.random.default_rng(0)
    a = np.eye(40) * 4 + rng.standard_normal((40, 40)) * 0.3
    b = rng.standard_normal(40)
    x, its, rel, ok = fgmres.fgmres(lambda v: a @ v, lambda v: v, b, rtol=1e-12)
    assert ok and its <= 40 and np.allclose(x, np.linalg.solve(a, b), rtol=1e-10)
    ainv = np.linalg.inv(a)
    x, its, rel, ok = fgmres.fgmres(lambda v: a @ v, lambda v: ainv @ v, b, rtol=1e-12)
    assert ok and its == 1
    x, its, rel, ok = fgmres.fgmres(lambda v: a @ v, lambda v: v, b, restart=3, rtol=1e-10, maxit=2000)
    assert ok and rel <= 1e-10 and np.allclose(x, np.linalg.solve(a, b), rtol=1e-8)


@pytest.mark.parametrize("dirichlet", [OUTFLOW2, si.ALL2])
def test_fgmres_vcycle_matches_direct_solve(dirichlet):
    spec = si.MeshSpec(2, (8, 4), (0.0, 0.0), (1.0, 0.5), 3, dirichlet)
    h = _hier(spec, 1)
    xs = si.reference_solution(spec, 1)
    b = h.apply(xs)
    x, its, rel, ok = fgmres.fgmres(h.apply, h.vcycle, b, rtol=1e-12)
    assert ok and rel <= 1e-12 and its < 30
    if spec.pure_dirichlet():
        x = multigrid.normalise_pressure(h.fine, x)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-7
