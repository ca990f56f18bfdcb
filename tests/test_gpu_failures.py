"""Failure detection without a GPU fault: the staged smoother's bounded waits report
STG_ETIMEOUT when their limit is set to zero (every wait gives up at once, the copies in
flight land, the kernel returns), the context stays usable afterwards, and non-finite
right-hand sides are rejected on the host."""
import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (12, 8), (0.0, 0.0), (2.2, 0.41), 3, OUT2)


def _pair(**opts):
    from paper_2210_02690_gb300 import Solver
    import oracle
    w = si.channel_w(SPEC, 1)
    gpu = Solver(SPEC, 1, 1e-3, 0.01, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, **opts)
    ref = oracle.Hierarchy(SPEC, 1, 1e-3, 0.01, w, newton=True, nu1=2, nu2=2)
    return gpu, ref


@pytest.mark.parametrize("use_graph", [1, 0])
def test_wait_limit_reports_timeout_and_context_recovers(use_graph):
    from paper_2210_02690_gb300 import StgError, set_wait_limit
    gpu, ref = _pair(use_graph=use_graph)
    b = ref.apply(si.reference_solution(SPEC, 1, seed=3))
    bt = torch.from_numpy(b).cuda()
    gpu.vcycle(bt)  # graph captured (when used) with the default limit
    set_wait_limit(0)
    try:
        with pytest.raises(StgError) as e:
            gpu.vcycle(bt)
        assert e.value.status == 6  # STG_ETIMEOUT
    finally:
        set_wait_limit(1 << 22)
    x = gpu.vcycle(bt).cpu().numpy()
    x_ref = ref.vcycle(b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-11
    gpu.close()


def test_non_finite_rhs_is_rejected():
    from paper_2210_02690_gb300 import StgError
    gpu, ref = _pair()
    b = torch.zeros(ref.fine.N, dtype=torch.float64, device="cuda")
    b[5] = float("nan")
    with pytest.raises(StgError) as e:
        gpu.gmres_solve(b)
    assert e.value.status == 1  # STG_EINVAL
    b[5] = 1.0
    x, its, rel, ok = gpu.gmres_solve(b)
    assert ok and rel <= 1e-8
    gpu.close()


def test_negative_wait_limit_is_rejected():
    from paper_2210_02690_gb300 import StgError, set_wait_limit
    with pytest.raises(StgError):
        set_wait_limit(-1)


def test_singular_local_matrix_reports_cell_and_context_recovers():
    """tau = 0 removes the pressure coupling of every local J_K (the velocity-pressure blocks carry
    the factor tau w_a): stg_setup and stg_set_slab_length return STG_ESINGULAR with a cell id; the
    live context is restored by a positive slab length and then matches the oracle again."""
    from paper_2210_02690_gb300 import Solver, StgError
    import oracle
    w = si.channel_w(SPEC, 1)
    for prec in (dict(), dict(vcycle_prec="f32", factor_prec="f32")):
        with pytest.raises(StgError) as e:
            Solver(SPEC, 1, 1e-3, 0.0, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, **prec)
        assert e.value.status == 4 and "cell" in str(e.value)
    gpu, ref = _pair()
    with pytest.raises(StgError) as e:
        gpu.set_slab_length(0.0)
    assert e.value.status == 4 and "cell" in str(e.value)
    with pytest.raises(StgError) as e:
        gpu.set_slab_length(float("nan"))
    assert e.value.status == 1
    gpu.set_slab_length(0.01)
    b = ref.apply(si.reference_solution(SPEC, 1, seed=3))
    x = gpu.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    x_ref = ref.vcycle(b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-12
    gpu.close()
    del oracle


def test_fgmres_iteration_limit_reports_noconv_with_results_written():
    """gmres_maxit = 1 at rtol 1e-14: STG_ENOCONV, with x (one preconditioned step) and the relative
    residual written; the context keeps working."""
    gpu, ref = _pair(gmres_maxit=1, gmres_rtol=1e-14)
    b = ref.apply(si.reference_solution(SPEC, 1, seed=4))
    bt = torch.from_numpy(b).cuda()
    x, its, relres, ok = gpu.gmres_solve(bt)
    assert not ok and its == 1
    x = x.cpu().numpy()
    true_rel = np.linalg.norm(b - ref.apply(x)) / np.linalg.norm(b)
    assert 1e-14 < relres < 1.0 and abs(relres - true_rel) <= 1e-6 * true_rel
    assert "gmres_maxit" in gpu.lib.stg_last_error(gpu.ctx).decode()
    x2, its2, rel2, ok2 = gpu.gmres_solve(bt, x0=torch.from_numpy(x).cuda())
    assert not ok2 and rel2 < relres            # a restart from the returned x keeps improving
    gpu.close()
