"""Parity of the GPU damped Newton (stg_newton_slab) and slab time march with the oracle (Sec. 3)."""
import numpy as np
import pytest

import stg_inputs as si
from oracle import mesh, newton

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (16, 8), (0.0, 0.0), (2.2, 0.41), 3, OUT2)
K, NU, TAU = 1, 1e-3, 0.02


def _setup():
    from paper_2210_02690_gb300 import Solver

    lev = mesh.Level(SPEC, SPEC.n_levels - 1, K)
    v0 = si.channel_w(SPEC, 0, pert=0.3)[0]
    g = np.repeat(si.channel_w(SPEC, 0, pert=0.0)[0][None], K + 1, axis=0)   # Poiseuille data
    X0 = np.zeros(lev.N)
    for a in range(K + 1):
        X0[a * (lev.R + lev.S):a * (lev.R + lev.S) + lev.R] = v0
    solver = Solver(SPEC, K, NU, TAU, torch.from_numpy(X0[:lev.R].repeat(K + 1)).cuda() * 0 +
                    torch.from_numpy(np.concatenate([v0] * (K + 1))).cuda(), nu1=2, nu2=2, gmres_rtol=1e-12)
    return solver, lev, v0, g, X0


def test_initial_residual_matches_oracle():
    solver, lev, v0, g, X0 = _setup()
    b = newton.rhs_nodal(lev, None, g, v0, NU, TAU)
    ref = np.linalg.norm(newton.residual(lev, X0, b, NU, TAU))
    _, steps, its, res, ok = solver.newton_slab(torch.from_numpy(X0).cuda(), v_prev=torch.from_numpy(v0).cuda(),
                                                g=torch.from_numpy(g.ravel()).cuda(), maxit=0)
    assert steps == 0 and abs(res - ref) <= 1e-12 * ref
    solver.close()


def test_newton_slab_matches_oracle():
    solver, lev, v0, g, X0 = _setup()
    b = newton.rhs_nodal(lev, None, g, v0, NU, TAU)
    X_ref, steps_ref, its_ref, hist = newton.newton_slab(SPEC, K, NU, TAU, X0, b, rtol=1e-10, gmres_rtol=1e-12)
    X, steps, its, res, ok = solver.newton_slab(torch.from_numpy(X0).cuda(), v_prev=torch.from_numpy(v0).cuda(),
                                                g=torch.from_numpy(g.ravel()).cuda(), rtol=1e-10)
    assert ok and steps == steps_ref
    assert abs(its - its_ref) <= steps
    X = X.cpu().numpy()
    assert np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref) < 1e-9
    assert res <= 1e-10 * hist[0] * 1.01
    solver.close()


def test_time_march_three_slabs():
    solver, lev, v0, g, X0 = _setup()
    Xo = X0.copy()
    vprev = v0.copy()
    Xg = torch.from_numpy(X0).cuda()
    vg = torch.from_numpy(v0).cuda()
    gg = torch.from_numpy(g.ravel()).cuda()
    for slab in range(3):
        b = newton.rhs_nodal(lev, None, g, vprev, NU, TAU)
        Xo, steps_ref, _, _ = newton.newton_slab(SPEC, K, NU, TAU, Xo, b, rtol=1e-10, gmres_rtol=1e-12)
        Xg, steps, _, _, ok = solver.newton_slab(Xg, v_prev=vg, g=gg, rtol=1e-10)
        assert ok and steps == steps_ref
        assert np.linalg.norm(Xg.cpu().numpy() - Xo) / np.linalg.norm(Xo) < 1e-9
        # next slab: previous end value as v_prev and as the initial guess at every Radau node
        vprev = newton.end_value(lev, Xo)
        Xo = np.concatenate([Xo.reshape(K + 1, -1)[-1]] * (K + 1))
        vg = Xg[K * (lev.R + lev.S):K * (lev.R + lev.S) + lev.R].clone()
        expect = np.concatenate([Xg.cpu().numpy().reshape(K + 1, -1)[-1]] * (K + 1))
        Xg = solver.slab_initial_guess(Xg)
        assert np.array_equal(Xg.cpu().numpy(), expect)
    solver.close()


def test_damped_newton_branch_matches_oracle():
    """The oracle's damping case (third full step raises ||F||, the half step is taken): the GPU
    takes the same number of steps to the same solution, so it damped the same step."""
    from test_oracle_newton import DAMP_K, DAMP_NU, DAMP_SPEC, DAMP_TAU, damping_case
    from paper_2210_02690_gb300 import Solver

    lev, b, X0, v0, g = damping_case()
    lams = []
    X_ref, steps_ref, _, hist = newton.newton_slab(DAMP_SPEC, DAMP_K, DAMP_NU, DAMP_TAU, X0, b, rtol=1e-10,
                                                   gmres_rtol=1e-12, lambdas=lams)
    assert min(lams) < 1.0
    w0 = torch.from_numpy(np.concatenate([X0[a * (lev.R + lev.S):a * (lev.R + lev.S) + lev.R]
                                          for a in range(DAMP_K + 1)])).cuda()
    solver = Solver(DAMP_SPEC, DAMP_K, DAMP_NU, DAMP_TAU, w0, nu1=2, nu2=2, gmres_rtol=1e-12)
    X, steps, its, res, ok = solver.newton_slab(torch.from_numpy(X0).cuda(), v_prev=torch.from_numpy(v0).cuda(),
                                                g=torch.from_numpy(g.ravel()).cuda(), rtol=1e-10)
    assert ok and steps == steps_ref
    X = X.cpu().numpy()
    assert np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref) < 1e-9
    solver.close()
