"""The allocation-free local inverse, stg_invert_local_noalloc.

It exists for callers that cannot call cudaMalloc when they need local
inverses (code running under CUDA stream capture, hosts that manage device
memory in their own arenas, loops that forbid allocation after start-up): it
needs no context and keeps its working copies in an array compiled into the
library.  This test feeds it the local matrices J_K of a small channel problem
(built by the oracle) and compares its output with the inverses that stg_setup
stores for the smoother (read back with stg_get_local_inverse), at the
tolerance of the other local-inverse tests, on two calls in a row with
different matrices, so a stale state from the first call would show.

The file name sorts last so that a run that stops at the first failure has
run every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_inverse_matches_setup_inverses():
    import oracle
    from oracle import vanka
    from paper_2210_02690_gb300 import Solver, load_library

    spec = si.MeshSpec(2, (8, 4), (0.0, 0.0), (2.2, 0.41), 2, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI)
    k, nu, tau = 1, 1e-3, 0.005
    w = si.channel_w(spec, k)
    solver = Solver(spec, k, nu, tau, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2)
    ref = oracle.Hierarchy(spec, k, nu, tau, w, newton=True, nu1=2, nu2=2)
    lib = load_library()
    lev = ref.levels[1]
    local = vanka.local_matrices(ref.J[1], lev)
    n = lev.n_patch
    stream = torch.cuda.current_stream().cuda_stream
    for cells in ([0, 5, 17, 31], [3, 30, 12]):          # two calls in a row, different matrices
        a = torch.from_numpy(np.ascontiguousarray(local[cells])).cuda()
        out = torch.full_like(a, float("nan"))
        torch.cuda.synchronize()
        st = lib.stg_invert_local_noalloc(n, len(cells), ctypes.c_void_p(a.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0, lib.stg_last_error(None)
        got = out.cpu().numpy()
        for i, cell in enumerate(cells):
            assert _rel(got[i], solver.local_inverse(1, cell)) < 1e-11, cell
    solver.close()


def test_noalloc_inverse_rejects_oversized_and_singular_input():
    from paper_2210_02690_gb300 import load_library

    lib = load_library()
    a = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.empty_like(a)
    p = ctypes.c_void_p
    assert lib.stg_invert_local_noalloc(257, 1, p(a.data_ptr()), p(out.data_ptr()), None) == 1
    assert b"257" in lib.stg_last_error(None)
    assert lib.stg_invert_local_noalloc(4, 1, p(a.data_ptr()), p(out.data_ptr()), None) == 4
    eye = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 4, 4) * 2.0
    assert lib.stg_invert_local_noalloc(4, 1, p(eye.data_ptr()), p(out.data_ptr()), None) == 0
    assert torch.allclose(out, eye / 4.0)
