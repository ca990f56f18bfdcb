"""Pins of the oracle's nonlinear slab residual F_n and damped Newton (Sec. 3, Eq. (3.2), (3.3))."""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, mesh, newton, timebasis

from test_oracle_assembly import NU, SPECS, T0, TAU, interpolant, pres_grad, traction_rhs, vel, vel_grad, vel_lap, vel_t


def _nodal(lev, fn, t_list):
    xn = lev.node_coords()
    return np.stack([fn(xn, t).ravel() for t in t_list])


def test_rhs_nodal_matches_rhs_for_exact_data():
    spec = SPECS["square_outflow"]
    lev = mesh.Level(spec, 0, 1)
    ts = T0 + TAU * timebasis.radau_nodes(1)
    f = lambda x, t: np.stack([x[:, 0] * x[:, 1] + t, x[:, 1] ** 2 - t * x[:, 0]], 1)   # in Q2
    g = lambda x, t: vel(x, t)
    vp = vel(lev.node_coords(), T0).ravel()
    ref = assemble.rhs_linear(lev, f, g, vp, NU, TAU, T0)
    got = newton.rhs_nodal(lev, _nodal(lev, f, ts), _nodal(lev, g, ts), vp, NU, TAU)
    assert np.linalg.norm(got - ref) < 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["square_outflow", "cube_dirichlet"])
def test_newton_jacobian_is_derivative_of_residual(name):
    lev = mesh.Level(SPECS[name], 0, 1)
    rng = np.random.default_rng(1)
    X = rng.standard_normal(lev.N)
    dX = rng.standard_normal(lev.N)
    b = rng.standard_normal(lev.N)
    eps = 1e-3
    fd = (newton.residual(lev, X + eps * dX, b, NU, TAU) - newton.residual(lev, X - eps * dX, b, NU, TAU)) / (2 * eps)
    jn = assemble.jacobian(lev, newton.velocity_part(lev, X), NU, TAU, newton=True)
    assert np.linalg.norm(fd - jn @ dX) < 1e-10 * np.linalg.norm(fd)


@pytest.mark.parametrize("name", ["square_dirichlet", "square_outflow", "cube_outflow"])
def test_nonlinear_manufactured_solution(name):
    # v quadratic in space, linear in time, p linear: the dG(k) solution of the Navier-Stokes slab
    # problem is its interpolant; f carries the nonlinear convection (v . grad) v
    spec = SPECS[name]
    k = 1
    lev = mesh.Level(spec, 0, k)

    def f(x, t):
        conv = np.einsum("ne,nce->nc", vel(x, t), vel_grad(x, t))
        return vel_t(x) + conv - NU * vel_lap(x, t) + pres_grad(x, t)

    b = assemble.rhs_linear(lev, f, lambda x, t: vel(x, t), vel(lev.node_coords(), T0).ravel(), NU, TAU, T0)
    b = b + traction_rhs(lev, NU, T0, TAU)
    X = interpolant(lev, T0, TAU)
    F = newton.residual(lev, X, b, NU, TAU)
    assert np.linalg.norm(F) < 1e-12 * np.linalg.norm(b)


def test_damped_newton_converges_quadratically():
    spec = si.MeshSpec(2, (8, 4), (0.0, 0.0), (2.2, 0.41), 2, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI)
    k, nu, tau = 1, 1e-3, 0.05
    lev = mesh.Level(spec, 1, k)
    v0 = si.channel_w(spec, 0)[0]
    g = np.repeat(si.channel_w(spec, 0, pert=0.0)[0][None], k + 1, axis=0)   # Poiseuille inflow/walls
    b = newton.rhs_nodal(lev, None, g, v0, nu, tau)
    X0 = np.zeros(lev.N)
    for a in range(k + 1):
        X0[a * (lev.R + lev.S):a * (lev.R + lev.S) + lev.R] = v0
    X, steps, its, hist = newton.newton_slab(spec, k, nu, tau, X0, b, rtol=1e-10, gmres_rtol=1e-12)
    assert hist[-1] <= 1e-10 * hist[0] and steps <= 8
    # quadratic convergence once close: the last contraction beats the square of the previous one
    r = np.array(hist) / hist[0]
    assert r[-1] < 1e3 * r[-2] ** 2 or r[-1] < 1e-13


# Damped-Newton data whose third full step raises ||F|| (ratio 1.40 against the sufficient-decrease
# bound) while the half step clears it (0.71): a single-level channel, so each linear solve is the
# exact coarse solve and the damping decision has wide margins on both sides.
DAMP_SPEC = si.MeshSpec(2, (8, 4), (0.0, 0.0), (2.2, 0.41), 1, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI)
DAMP_K, DAMP_NU, DAMP_TAU, DAMP_SCALE = 1, 1e-2, 0.5, 20.0


def damping_case():
    """(level, right-hand side, initial guess 20x the Poiseuille-plus-perturbation field)."""
    lev = mesh.Level(DAMP_SPEC, 0, DAMP_K)
    v0 = si.channel_w(DAMP_SPEC, 0)[0]
    g = np.repeat(si.channel_w(DAMP_SPEC, 0, pert=0.0)[0][None], DAMP_K + 1, axis=0)
    b = newton.rhs_nodal(lev, None, g, v0, DAMP_NU, DAMP_TAU)
    X0 = np.zeros(lev.N)
    for a in range(DAMP_K + 1):
        X0[a * (lev.R + lev.S):a * (lev.R + lev.S) + lev.R] = DAMP_SCALE * v0
    return lev, b, X0, v0, g


def test_damped_newton_takes_the_largest_admissible_step():
    """Reading A23: lambda is the first of 1, 1/2, .., 1/16 with ||F(X + lambda C)|| < (1 - 1e-4 lambda)
    ||F(X)||.  The check re-runs every step from the accepted iterates, evaluates all five candidates
    with the exact direction (one-level hierarchy: the preconditioned solve is exact) and asks for the
    largest admissible one; at least one step must be damped."""
    from oracle import fgmres, multigrid
    lev, b, X0, _, _ = damping_case()
    lams = []
    X, steps, its, hist = newton.newton_slab(DAMP_SPEC, DAMP_K, DAMP_NU, DAMP_TAU, X0, b, rtol=1e-10,
                                             gmres_rtol=1e-12, lambdas=lams)
    assert hist[-1] <= 1e-10 * hist[0] and steps == len(lams)
    assert min(lams) < 1.0
    Xm = X0.copy()
    cand = [2.0 ** -i for i in range(5)]
    for lam in lams:
        F = newton.residual(lev, Xm, b, DAMP_NU, DAMP_TAU)
        jac = assemble.jacobian(lev, newton.velocity_part(lev, Xm), DAMP_NU, DAMP_TAU, newton=True)
        C = np.linalg.solve(jac.toarray(), -F)
        fn = np.linalg.norm(F)
        ok = [np.linalg.norm(newton.residual(lev, Xm + c * C, b, DAMP_NU, DAMP_TAU)) < (1 - 1e-4 * c) * fn
              for c in cand]
        expect = next((c for c, o in zip(cand, ok) if o), cand[-1])
        assert lam == expect
        if lam < 1.0:
            assert not ok[0]                     # the full step would have raised the residual
        Xm = Xm + lam * C
    assert np.linalg.norm(Xm - X) <= 1e-10 * np.linalg.norm(X)
    del fgmres, multigrid


def test_damping_floor_accepts_lambda_min():
    """With lambda_min = 1 every step is the full step, also the one that raises ||F||: the floor
    branch accepts lambda_min when no candidate decreases enough."""
    lev, b, X0, _, _ = damping_case()
    lams = []
    _, steps, _, hist = newton.newton_slab(DAMP_SPEC, DAMP_K, DAMP_NU, DAMP_TAU, X0, b, rtol=1e-10,
                                           gmres_rtol=1e-12, lambdas=lams, lam_min=1.0, maxit=4)
    assert lams == [1.0] * 4
    assert hist[3] > hist[2]                     # the undamped third step raised the residual
