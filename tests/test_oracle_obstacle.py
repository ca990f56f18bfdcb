"""Pins of the oracle's obstacle domain: cells of a box removed from the mesh, Nitsche's Dirichlet
terms (Eq. (2.1)) on the faces of the remaining cells that border it, identity rows for the
unknowns left without an equation (velocity at Q2 nodes of removed cells only, pressure of
removed cells).

* Galerkin exactness: the manufactured quadratic velocity / linear pressure of
  test_oracle_assembly, with its values as Dirichlet data on every Dirichlet face including the
  obstacle's and zero at the unknowns without an equation, solves the discrete slab problem to
  rounding (2D, k = 0, 1, 2, an outflow and an all-Dirichlet box; Oseen and Newton).  A missing or
  mis-signed obstacle face term, a wrong normal or a coupling into the removed unknowns breaks it.
* Structure: removed unknowns are decoupled identity rows and columns; the obstacle face list
  matches the geometry (each listed face's neighbour cell lies in the box).
"""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, mesh

from test_oracle_assembly import NU, T0, TAU, forcing, interpolant, nodal_w, traction_rhs, vel

SPECS = {
    "box_outflow": si.MeshSpec(2, (8, 8), (0.0, 0.0), (1.6, 1.0), 2, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI,
                               (1, 2, 1, 3)),
    "box_dirichlet": si.MeshSpec(2, (8, 4), (0.1, 0.0), (1.7, 0.8), 2, si.ALL2, (2, 3, 1, 2)),
}


def manufactured(spec, k, newton=False):
    lev = mesh.Level(spec, spec.n_levels - 1, k)
    jac = assemble.jacobian(lev, nodal_w(lev), NU, TAU, newton=newton)
    x = interpolant(lev, T0, TAU)
    x[assemble.dead_dofs(lev)] = 0.0
    vprev = vel(lev.node_coords(), T0).ravel()
    vprev.reshape(-1, 2)[lev.dead_nodes] = 0.0
    b = assemble.rhs_linear(lev, forcing(NU), lambda xx, t: vel(xx, t), vprev, NU, TAU, T0)
    b = b + traction_rhs(lev, NU, T0, TAU)
    return lev, jac, x, b


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("k", [0, 1, 2])
def test_obstacle_galerkin_exactness(name, k):
    lev, jac, x, b = manufactured(SPECS[name], k)
    assert lev.masked.sum() > 0 and len(lev.dead_nodes) > 0
    assert np.linalg.norm(jac @ x - b) < 1e-12 * np.linalg.norm(b)


def test_obstacle_faces_are_needed():
    """Without the obstacle's face terms the manufactured solution no longer solves the problem."""
    spec = SPECS["box_outflow"]
    lev, jac, x, b = manufactured(spec, 1)
    # only the domain's Dirichlet faces (of the remaining cells): the obstacle's are dropped
    domain = [(e, side, c[~lev.masked[c]]) for e, side, c in lev.boundary_faces() if lev.is_dirichlet(e, side)]
    lev.dirichlet_faces = lambda: domain
    jac2 = assemble.jacobian(lev, nodal_w(lev), NU, TAU, newton=False)
    assert np.linalg.norm(jac2 @ x - b) > 1e-6 * np.linalg.norm(b)


@pytest.mark.parametrize("name", list(SPECS))
def test_removed_unknowns_are_decoupled_identity_rows(name):
    lev, jac, _, _ = manufactured(SPECS[name], 1, newton=True)
    dead = assemble.dead_dofs(lev)
    live = np.setdiff1d(np.arange(lev.N), dead)
    j = jac.tocsr()
    assert np.array_equal(j[dead][:, dead].toarray(), np.eye(len(dead)))
    assert j[live][:, dead].nnz == 0 and j[dead][:, live].nnz == 0


def test_obstacle_faces_match_geometry():
    lev = mesh.Level(SPECS["box_outflow"], 1, 0)
    box = SPECS["box_outflow"].obstacle_cells(1)
    assert box == (2, 4, 2, 6)
    count = 0
    for e, side, cells in lev.dirichlet_faces():
        for c in cells:
            ij = lev.cell_idx[c].copy()
            assert not lev.masked[c]
            ij[e] += 1 if side else -1
            if 0 <= ij[e] < lev.cells[e]:
                nb = ij[0] + lev.cells[0] * ij[1]
                assert lev.masked[nb]
                count += 1
    assert count == 2 * (box[1] - box[0]) + 2 * (box[3] - box[2])


def test_obstacle_prolongation_reproduces_fluid_functions():
    """P maps a coarse FE function of the fluid domain to the same function on the fine mesh (the
    fine unknowns outside the domain are zero, so R = P^T carries no residual from them)."""
    from oracle import transfer
    spec = SPECS["box_outflow"]
    coarse, fine = mesh.Level(spec, 0, 1), mesh.Level(spec, 1, 1)
    P = transfer.prolongation(coarse, fine)
    xc = np.random.default_rng(3).standard_normal(coarse.N)
    xc[assemble.dead_dofs(coarse)] = 0.0
    xf = P @ xc
    dead = assemble.dead_dofs(fine)
    assert np.all(xf[dead] == 0.0)
    plain = transfer.prolongation(coarse, fine.__class__(si.MeshSpec(2, spec.n, spec.lo, spec.hi, spec.n_levels,
                                                                      spec.dirichlet), 1, 1))
    live = np.setdiff1d(np.arange(fine.N), dead)
    assert np.allclose(xf[live], (plain @ xc)[live], atol=1e-14)
    assert P[:, assemble.dead_dofs(coarse)].nnz == 0


def test_obstacle_multigrid_keeps_its_iteration_count():
    """FGMRES with the V-cycle on a channel with an interior obstacle needs about as many iterations
    as without one (7 here); transfers that let the residual of the removed unknowns into the
    coarse problem raise it to about 50."""
    import oracle
    from oracle import fgmres
    out2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
    its = {}
    for obst in ((), (3, 5, 3, 5)):
        spec = si.MeshSpec(2, (88, 16), (0.0, 0.0), (2.2, 0.41), 2, out2, obst)
        w = si.channel_w(spec, 1)
        h = oracle.Hierarchy(spec, 1, 1e-3, 0.005, w, newton=True, nu1=2, nu2=2)
        xs = si.reference_solution(spec, 1)
        xs[assemble.dead_dofs(h.fine)] = 0.0
        b = h.apply(xs)
        _, its[obst], _, ok = fgmres.fgmres(h.apply, h.vcycle, b)
        assert ok
    assert its[(3, 5, 3, 5)] <= its[()] + 3, its


@pytest.mark.parametrize("k", [0, 1])
def test_forces_of_quadratic_fields_equal_the_volume_integral(k):
    """For v quadratic and p linear (the manufactured fields), the surface integral equals
    int_O (nu Laplace v - grad p) dV by the divergence theorem (the face rule is exact), evaluated
    at each Radau node; the sign (force on the obstacle) and both components are checked."""
    from oracle import functionals, timebasis
    from test_oracle_assembly import pres_grad, vel_lap
    spec = SPECS["box_outflow"]
    lev = mesh.Level(spec, 1, k)
    x = interpolant(lev, T0, TAU)
    F = functionals.obstacle_forces(lev, x, NU)
    box = spec.obstacle_cells(1)
    area = (box[1] - box[0]) * lev.h[0] * (box[3] - box[2]) * lev.h[1]
    for a, c in enumerate(timebasis.radau_nodes(k)):
        t = T0 + TAU * c
        pt = np.zeros((1, 2))
        expect = area * (NU * vel_lap(pt, t)[0] - pres_grad(pt, t)[0])
        assert np.allclose(F[a], expect, rtol=1e-12, atol=1e-14), (F[a], expect)


def test_uniform_pressure_exerts_no_force_and_sign_of_front_pressure():
    from oracle import functionals
    spec = SPECS["box_outflow"]
    lev = mesh.Level(spec, 1, 0)
    x = np.zeros(lev.N)
    x[lev.pres_index(0, np.arange(lev.n_cells), 0)] = 3.0
    assert np.allclose(functionals.obstacle_forces(lev, x, NU), 0.0, atol=1e-14)
    # pressure decreasing downstream pushes the obstacle downstream (+x drag)
    cen = lev.cell_centres()
    x[lev.pres_index(0, np.arange(lev.n_cells), 0)] = -cen[:, 0]
    x[lev.pres_index(0, np.arange(lev.n_cells), 1)] = -lev.h[0] / 2
    F = functionals.obstacle_forces(lev, x, NU)
    assert F[0, 0] > 0 and abs(F[0, 1]) < 1e-14
