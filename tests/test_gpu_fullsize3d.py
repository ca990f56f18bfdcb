"""Parity at the full size of the 3D workload (unit cube 48^3, dG(1), 170 x 170 local matrices,
levels 6^3 .. 48^3, FP32 factors and V-cycle, FP64 outer FGMRES), on sampled outputs the oracle
computes one by one from 3x3x3-cell window meshes (window.py, pinned in 2D and 3D by
test_oracle_window.py): the FP32 J_K^{-1} of interior, face, edge and corner cells, the rows of
J x at their patches, and the FGMRES true residual of the whole system.
"""
import numpy as np
import pytest

import stg_inputs as si
from window import window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG = si.WORKLOADS["cube48_k1"]
SPEC, K = CFG["spec"], CFG["k"]
N1 = SPEC.n[0]
EPS = np.finfo(float).eps
SAMPLES = [(24, 20, 17), (0, 30, 11), (47, 5, 40), (13, 0, 47), (0, 0, 25), (47, 47, 47), (0, 47, 0), (46, 1, 2)]


@pytest.fixture(scope="module")
def w_full():
    return si.fourier_w(SPEC, K, seed=si.BASE_SEED)


@pytest.fixture(scope="module")
def gpu32(w_full):
    from paper_2210_02690_gb300 import Solver
    s = Solver(SPEC, K, CFG["nu"], CFG["tau"], torch.from_numpy(w_full.ravel()).cuda(), nu1=CFG["nu1"],
               nu2=CFG["nu2"], linearisation="oseen", vcycle_prec="f32", factor_prec="f32")
    yield s
    s.close()


def _cell(c):
    return c[0] + N1 * (c[1] + N1 * c[2])


def test_local_inverse_and_rows_full_size_3d(w_full, gpu32):
    n = si.n_dofs(3, SPEC.n, K)
    x = si.random_vector(n, 77)
    y = gpu32.apply_jacobian(torch.from_numpy(x).cuda()).cpu().numpy()
    top = SPEC.n_levels - 1
    for c in SAMPLES:
        lev, J, gidx, dofs = window(SPEC, K, w_full, *c, nu=CFG["nu"], tau=CFG["tau"], newton=False)
        JK = J[np.ix_(dofs, dofs)]
        inv = np.linalg.inv(JK)
        cond = np.linalg.cond(JK)
        g32 = gpu32.local_inverse(top, _cell(c))
        assert np.linalg.norm(g32 - inv) / np.linalg.norm(inv) < 50 * cond * 6e-8, c
        xw = x[gidx]
        rows = J[dofs] @ xw
        bound = 64 * EPS * (np.abs(J[dofs]) @ np.abs(xw))
        assert np.all(np.abs(y[gidx[dofs]] - rows) <= bound + 1e-300), c


def test_fgmres_true_residual_full_size_3d(gpu32):
    xs = torch.from_numpy(si.reference_solution(SPEC, K, seed=si.BASE_SEED + 1)).cuda()
    b = gpu32.apply_jacobian(xs)
    x, its, rel, ok = gpu32.gmres_solve(b)
    assert ok and rel <= 1e-8 and its <= 10
    r = b - gpu32.apply_jacobian(x)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1.01e-8
