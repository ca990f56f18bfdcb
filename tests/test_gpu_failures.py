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
