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
