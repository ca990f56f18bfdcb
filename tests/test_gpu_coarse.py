"""Accuracy of the coarse direct solve (Sec. 3: a direct solver on T_0) on the coarse level of the
bench workload: the 88x16 channel, dG(1), Newton Jacobian, 31 812 unknowns.

* FP64 factors (the FP64 form, with its default one step of iterative refinement): the normwise
  backward error eta = ||b - J x||_inf / (||J||_inf ||x||_inf + ||b||_inf) of the solve, at the
  level of an LU solve with partial pivoting; without the refinement step, the explicit block
  inverses of the cyclic reduction leave a relative residual below 1e-13.
* FP32 factors (the F32 form's default): the relative residual after 0, 1 and 2 steps of iterative
  refinement with FP64 residuals; each step contracts it by about cond(J_0) u_32.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import stg_inputs as si
from oracle import assemble, mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (88, 16), (0.0, 0.0), (2.2, 0.41), 1, OUT2)
K, NU, TAU = 1, 1e-3, 0.005


@pytest.fixture(scope="module")
def data():
    w = si.channel_w(SPEC, K)
    lev = mesh.Level(SPEC, 0, K)
    J = assemble.jacobian(lev, w, NU, TAU, newton=True).tocsr()
    b = J @ si.reference_solution(SPEC, K, seed=5)
    return w, J, b


def _eta(J, x, b):
    r = b - J @ x
    return np.max(np.abs(r)) / (spla.norm(J, np.inf) * np.max(np.abs(x)) + np.max(np.abs(b)))


def test_fp64_coarse_solve_backward_error(data):
    from paper_2210_02690_gb300 import Solver
    w, J, b = data
    for steps, eta_bar, rel_bar in ((1, 1e-15, 1e-14), (0, 2e-14, 1e-13)):
        s = Solver(SPEC, K, NU, TAU, torch.from_numpy(w.ravel()).cuda(), coarse_refine=steps)
        x = s.coarse_solve(torch.from_numpy(b).cuda()).cpu().numpy()
        eta = _eta(J, x, b)
        rel = np.linalg.norm(b - J @ x) / np.linalg.norm(b)
        assert eta < eta_bar and rel < rel_bar, (steps, eta, rel)
        s.close()


def test_fp32_coarse_refinement_contracts(data):
    from paper_2210_02690_gb300 import Solver
    w, J, b = data
    res = []
    for steps in (0, 1, 2):
        s = Solver(SPEC, K, NU, TAU, torch.from_numpy(w.ravel()).cuda(), vcycle_prec="f32", factor_prec="f32",
                   coarse_prec="f32", coarse_refine=steps)
        x = s.coarse_solve(torch.from_numpy(b).cuda()).cpu().numpy()
        res.append(np.linalg.norm(b - J @ x) / np.linalg.norm(b))
        s.close()
    # FP32 factors alone: about cond u_32; each refinement step multiplies by about cond u_32
    assert res[0] < 1e-3, res
    assert res[1] < 1e-2 * res[0] and res[2] < 1e-2 * res[1], res
