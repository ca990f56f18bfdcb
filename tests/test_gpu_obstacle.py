"""Parity of the CUDA path with the oracle on a channel with an obstacle (cells of a box removed;
no-slip Nitsche faces around it; identity rows for the unknowns outside the fluid domain; the
removed cells' patches smooth only those; transfers of the fluid domain; the coarse solver with a
second pressure group for the cell columns the obstacle splits), the Newton time march on it and
the drag and lift forces (Sec. 4's benchmark quantities, surface integrals over the obstacle)."""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, fgmres, functionals, mesh, newton, vanka

from test_gpu_parity import FP64_BAR, brel, brel_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (64, 16), (0.0, 0.0), (2.2, 0.41), 3, OUT2, (3, 5, 1, 3))
K, NU, TAU = 1, 1e-3, 0.01
EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def pair():
    import oracle
    from paper_2210_02690_gb300 import Solver
    w = si.obstacle_inflow(SPEC, K) + si.channel_w(SPEC, K, u_max=0.0, pert=0.3)
    gpu = Solver(SPEC, K, NU, TAU, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, gmres_rtol=1e-12)
    ref = oracle.Hierarchy(SPEC, K, NU, TAU, w, newton=True, nu1=2, nu2=2)
    yield gpu, ref
    gpu.close()


def _rhs(ref, seed=7):
    xs = si.reference_solution(SPEC, K, seed=seed)
    xs[assemble.dead_dofs(ref.fine)] = 0.0
    return ref.apply(xs)


def test_operators_and_local_inverses(pair):
    gpu, ref = pair
    for lvl, lev in enumerate(ref.levels):
        x = si.random_vector(lev.N, 11 + lvl)
        y = gpu.apply_jacobian(torch.from_numpy(x).cuda(), level=lvl).cpu().numpy()
        y_ref = ref.J[lvl] @ x
        bound = 64 * EPS * np.linalg.norm(abs(ref.J[lvl]) @ np.abs(x)) / np.linalg.norm(y_ref)
        assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < bound, lvl
        if lvl == 0:
            continue
        cells = [0, lev.n_cells - 1] + list(np.nonzero(lev.masked)[0][:2])
        box = SPEC.obstacle_cells(lvl)
        cells += [box[2] * lev.cells[0] + box[0] - 1, (box[3]) * lev.cells[0] + box[0]]  # next to it
        for cell in cells:
            g = gpu.local_inverse(lvl, int(cell))
            assert brel_matrix(g, ref.jinv[lvl][cell], lev) < 1e-11, (lvl, cell)


def test_transfers(pair):
    gpu, ref = pair
    for lvl in range(1, len(ref.levels)):
        xc = si.random_vector(ref.levels[lvl - 1].N, 3)
        xf = si.random_vector(ref.levels[lvl].N, 4)
        p = gpu.prolongate(lvl, torch.from_numpy(xc).cuda(), torch.from_numpy(xf).cuda()).cpu().numpy()
        assert np.linalg.norm(p - xf - ref.P[lvl] @ xc) < 1e-14 * np.linalg.norm(p)
        r = gpu.restrict(lvl, torch.from_numpy(xf).cuda()).cpu().numpy()
        assert np.linalg.norm(r - ref.P[lvl].T @ xf) < 1e-14 * np.linalg.norm(r)


def test_coarse_solve_sweep_and_vcycle(pair):
    gpu, ref = pair
    lev0 = ref.levels[0]
    xs = si.reference_solution(SPEC, K, seed=5, level=0)
    b0 = ref.J[0] @ xs
    x0 = gpu.coarse_solve(torch.from_numpy(b0).cuda()).cpu().numpy()
    assert np.linalg.norm(ref.J[0] @ x0 - b0) < 1e-13 * np.linalg.norm(b0)
    assert np.linalg.norm(x0 - ref.coarse_solve(b0)) < 1e-10 * np.linalg.norm(x0)
    lvl = len(ref.levels) - 1
    lev = ref.levels[lvl]
    b = si.random_vector(lev.N, 21)
    d0 = si.random_vector(lev.N, 22)
    d = gpu.smooth(lvl, 3, torch.from_numpy(b).cuda(), torch.from_numpy(d0).cuda()).cpu().numpy()
    d_ref = vanka.sweep_averaged(ref.J[lvl], lev, ref.jinv[lvl], b, d0, 0.7, 3)
    assert brel(d, d_ref, lev) < FP64_BAR
    bb = _rhs(ref)
    v = gpu.vcycle(torch.from_numpy(bb).cuda()).cpu().numpy()
    assert brel(v, ref.vcycle(bb), ref.fine) < FP64_BAR
    del lev0


def test_fgmres_iterations_match_oracle(pair):
    gpu, ref = pair
    b = _rhs(ref)
    x, its, rel, ok = gpu.gmres_solve(torch.from_numpy(b).cuda())
    _, its_ref, _, ok_ref = fgmres.fgmres(ref.apply, ref.vcycle, b, rtol=1e-12)
    assert ok and ok_ref and abs(its - its_ref) <= 1, (its, its_ref)
    assert np.linalg.norm(b - ref.apply(x.cpu().numpy())) <= 2e-12 * np.linalg.norm(b)


def test_f32_form_on_the_obstacle_channel():
    import oracle
    from paper_2210_02690_gb300 import Solver
    w = si.obstacle_inflow(SPEC, K)
    gpu = Solver(SPEC, K, NU, TAU, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, vcycle_prec="f32",
                 factor_prec="f32")
    ref = oracle.Hierarchy(SPEC, K, NU, TAU, w, newton=True, nu1=2, nu2=2)
    b = _rhs(ref)
    v = gpu.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    x_ref = ref.vcycle(b)
    assert np.linalg.norm(v - x_ref) / np.linalg.norm(x_ref) < 1e-4
    x, its, rel, ok = gpu.gmres_solve(torch.from_numpy(b).cuda())
    _, its_ref, _, _ = fgmres.fgmres(ref.apply, ref.vcycle, b, rtol=1e-8)
    assert ok and its <= its_ref + 1
    gpu.close()


def test_newton_march_and_forces_match_oracle():
    """Three slabs of the Newton time march from rest with the Poiseuille inflow (the impulsive
    start of Sec. 4): the same Newton steps as the oracle, the same slab solutions, and drag and
    lift at every Radau node equal to the oracle's surface integrals."""
    from paper_2210_02690_gb300 import Solver
    lev = mesh.Level(SPEC, SPEC.n_levels - 1, K)
    g = si.obstacle_inflow(SPEC, K)
    X0 = np.zeros(lev.N)
    solver = Solver(SPEC, K, NU, TAU, torch.from_numpy(np.zeros((K + 1) * lev.R)).cuda(), nu1=2, nu2=2,
                    gmres_rtol=1e-12)
    Xo, vprev = X0.copy(), np.zeros(lev.R)
    Xg, vg, gg = torch.from_numpy(X0).cuda(), torch.zeros(lev.R, dtype=torch.float64).cuda(), \
        torch.from_numpy(g.ravel()).cuda()
    for slab in range(3):
        b = newton.rhs_nodal(lev, None, g, vprev, NU, TAU)
        Xo, steps_ref, _, _ = newton.newton_slab(SPEC, K, NU, TAU, Xo, b, rtol=1e-10, gmres_rtol=1e-12)
        Xg, steps, _, _, ok = solver.newton_slab(Xg, v_prev=vg, g=gg, rtol=1e-10)
        assert ok and steps == steps_ref, (slab, steps, steps_ref)
        Xh = Xg.cpu().numpy()
        assert np.linalg.norm(Xh - Xo) / np.linalg.norm(Xo) < 1e-9
        F = solver.obstacle_forces(Xg)
        F_ref = functionals.obstacle_forces(lev, Xo, NU)
        assert np.allclose(F, F_ref, rtol=1e-8, atol=1e-12 * np.abs(F_ref).max()), (F, F_ref)
        vprev = newton.end_value(lev, Xo)
        Xo = np.concatenate([Xo.reshape(K + 1, -1)[-1]] * (K + 1))
        vg = Xg[K * (lev.R + lev.S):K * (lev.R + lev.S) + lev.R].clone()
        Xg = solver.slab_initial_guess(Xg)
    assert F_ref[-1, 0] > 0           # the flow drags the obstacle downstream
    solver.close()


def test_invalid_obstacles_are_rejected():
    from paper_2210_02690_gb300 import Solver, StgError
    for ob in ((0, 16, 1, 2), (3, 2, 1, 2), (3, 5, 1, 9)):
        spec = si.MeshSpec(2, (64, 16), (0.0, 0.0), (2.2, 0.41), 3, OUT2, ob)
        with pytest.raises(StgError) as e:
            Solver(spec, K, NU, TAU, torch.zeros((K + 1) * 2 * 129 * 33, dtype=torch.float64).cuda())
        assert e.value.status == 1
