"""Parity at the full size of the bench workload (2D channel 704x128, dG(1), Newton Jacobian,
4 levels), in the launch configuration bench.py times (autotuned colour kernels), on sampled
outputs the oracle can compute one by one (J_K^{-1} and the rows of J x at sampled cells, from
window meshes: see window.py, pinned by test_oracle_window.py), on one FP64 V-cycle against the
oracle's V-cycle of the whole channel (about a minute of oracle set-up), plus properties that
hold at any size.
"""
import numpy as np
import pytest

import stg_inputs as si
from test_gpu_parity import FP64_BAR, brel, brel_matrix
from window import window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG = si.WORKLOADS["channel704_k1"]
SPEC, K = CFG["spec"], CFG["k"]
NX, NY = SPEC.n
H = ((SPEC.hi[0] - SPEC.lo[0]) / NX, (SPEC.hi[1] - SPEC.lo[1]) / NY)
EPS = np.finfo(float).eps
# interior, inflow wall, both walls, outflow, corners
SAMPLES = [(350, 60), (0, 64), (400, 0), (123, NY - 1), (NX - 1, 77), (0, 0), (NX - 1, NY - 1), (NX - 2, 1)]


@pytest.fixture(scope="module")
def w_full():
    return si.channel_w(SPEC, K, seed=si.BASE_SEED)


def _solver(w, **form):
    from paper_2210_02690_gb300 import Solver
    return Solver(SPEC, K, CFG["nu"], CFG["tau"], torch.from_numpy(w.ravel()).cuda(), nu1=CFG["nu1"],
                  nu2=CFG["nu2"], linearisation="newton", **form)


@pytest.fixture(scope="module")
def gpu64(w_full):
    s = _solver(w_full)
    s.autotune()
    yield s
    s.close()


@pytest.fixture(scope="module")
def gpu32(w_full):
    s = _solver(w_full, vcycle_prec="f32", factor_prec="f32")
    s.autotune()
    yield s
    s.close()


@pytest.fixture(scope="module")
def gpubf16(w_full):
    s = _solver(w_full, vcycle_prec="f32", factor_prec="bf16")
    s.autotune()
    yield s
    s.close()


def _window(cx, cy, w_full):
    return window(SPEC, K, w_full, cx, cy, nu=CFG["nu"], tau=CFG["tau"])


@pytest.mark.parametrize("cell", SAMPLES)
def test_local_inverse_full_size(cell, w_full, gpu64, gpu32):
    cx, cy = cell
    lev, J, gidx, dofs = _window(cx, cy, w_full)
    JK = J[np.ix_(dofs, dofs)]
    inv = np.linalg.inv(JK)
    cond = np.linalg.cond(JK)
    top = SPEC.n_levels - 1
    g64 = gpu64.local_inverse(top, cy * NX + cx)
    assert brel_matrix(g64, inv, lev) < FP64_BAR
    # FP32 factors from the equilibrated FP32 J_K: rounding u = 6e-8 amplified by cond(J_K)
    g32 = gpu32.local_inverse(top, cy * NX + cx)
    assert np.linalg.norm(g32 - inv) / np.linalg.norm(inv) < 50 * cond * 6e-8


def test_operator_rows_full_size(w_full, gpu64):
    n = si.n_dofs(2, SPEC.n, K)
    x = si.random_vector(n, 77)
    y = gpu64.apply_jacobian(torch.from_numpy(x).cuda()).cpu().numpy()
    for cx, cy in SAMPLES:
        lev, J, gidx, dofs = _window(cx, cy, w_full)
        xw = x[gidx]
        rows = J[dofs] @ xw
        bound = 64 * EPS * (np.abs(J[dofs]) @ np.abs(xw))
        assert np.all(np.abs(y[gidx[dofs]] - rows) <= bound + 1e-300), (cx, cy)


@pytest.mark.parametrize("form", ["gpu64", "gpu32"])
def test_vcycle_is_linear_full_size(form, request):
    """V(b1 + 2 b2) = V(b1) + 2 V(b2) up to rounding: the V-cycle is a fixed linear operator."""
    s = request.getfixturevalue(form)
    n = si.n_dofs(2, SPEC.n, K)
    b1 = torch.from_numpy(si.random_vector(n, 5)).cuda()
    b2 = torch.from_numpy(si.random_vector(n, 6)).cuda()
    v1, v2 = s.vcycle(b1).clone(), s.vcycle(b2).clone()
    v12 = s.vcycle(b1 + 2 * b2)
    tol = 1e-12 if form == "gpu64" else 1e-5
    assert float(torch.linalg.norm(v12 - v1 - 2 * v2) / torch.linalg.norm(v12)) < tol


@pytest.mark.parametrize("form", ["gpu64", "gpu32", "gpubf16"])
def test_fgmres_true_residual_full_size(form, request, gpu64):
    """FGMRES stops at 1e-8 relative, checked with the FP64 operator (same on every form); the
    reduced-precision forms need at most one iteration more than the FP64 form."""
    s = request.getfixturevalue(form)
    xs = torch.from_numpy(si.reference_solution(SPEC, K, seed=si.BASE_SEED + 1)).cuda()
    b = gpu64.apply_jacobian(xs)
    x, its, rel, ok = s.gmres_solve(b)
    assert ok and rel <= 1e-8 and its <= 8
    r = b - gpu64.apply_jacobian(x)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1.01e-8
    _, its64, _, _ = gpu64.gmres_solve(b)
    assert its <= its64 + 1


def test_fp64_vcycle_full_size_matches_oracle(w_full, gpu64):
    """One FP64 V-cycle of the whole 704x128 channel against the oracle's, block by block."""
    import oracle
    ref = oracle.Hierarchy(SPEC, K, CFG["nu"], CFG["tau"], w_full, newton=True, nu1=CFG["nu1"], nu2=CFG["nu2"])
    b = ref.apply(si.reference_solution(SPEC, K, seed=si.BASE_SEED + 1))
    x = gpu64.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    x_ref = ref.vcycle(b)
    err = brel(x, x_ref, ref.fine)
    assert err < FP64_BAR, err
