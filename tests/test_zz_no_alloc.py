"""The allocation-free local inverse, stg_invert_local_noalloc.

It exists for callers that cannot call cudaMalloc when they need local
inverses: host applications that own the GPU's memory and hand it out only
from their own pools, and real-time loops that forbid allocation after
start-up.  It needs no context and keeps its working copies in an 8 MiB array
compiled into the library (2^20 doubles, so at most 2^20 / n^2 matrices per
launch).  These tests compare its output with the inverses that stg_setup
stores for the smoother (two calls in a row with different matrices, so a
stale state from the first call would show), with numpy.linalg.inv on counts
that need several launches over the shared array and at the largest order
n = 256, and check that a call with two singular matrices reports the lower
index.

The file name sorts last so that a run that stops at the first failure has
run every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCRATCH_DOUBLES = 1 << 20


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _call(lib, n, a, out, stream=None):
    p = ctypes.c_void_p
    return lib.stg_invert_local_noalloc(n, a.shape[0], p(a.data_ptr()), p(out.data_ptr()),
                                        p(stream) if stream is not None else None)


def _well_conditioned(rng, count, n):
    # diagonally dominant with random signs and permuted rows: pivoting is exercised, cond stays small
    a = rng.standard_normal((count, n, n))
    a += np.eye(n)[None] * (2.0 * n ** 0.5) * rng.choice([-1.0, 1.0], size=(count, 1, n))
    perm = np.stack([rng.permutation(n) for _ in range(count)])
    return np.take_along_axis(a, perm[:, :, None], axis=1)


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
        st = _call(lib, n, a, out, stream)
        assert st == 0, lib.stg_last_error(None)
        got = out.cpu().numpy()
        for i, cell in enumerate(cells):
            assert _rel(got[i], solver.local_inverse(1, cell)) < 1e-11, cell
            assert _rel(got[i], ref.jinv[1][cell]) < 1e-11, cell
    solver.close()


@pytest.mark.parametrize("n, count", [(42, 700), (256, 40)])
def test_noalloc_inverse_against_lapack_over_several_launches(n, count):
    """count > 2^20 / n^2: the call runs several launches that reuse the shared scratch array."""
    from paper_2210_02690_gb300 import load_library

    lib = load_library()
    assert count > SCRATCH_DOUBLES // (n * n)
    rng = np.random.default_rng(1000 + n)
    for call in range(2):
        a_h = _well_conditioned(rng, count, n)
        a = torch.from_numpy(a_h).cuda()
        out = torch.full_like(a, float("nan"))
        assert _call(lib, n, a, out) == 0, lib.stg_last_error(None)
        got = out.cpu().numpy()
        ref = np.linalg.inv(a_h)
        err = max(_rel(g, r) for g, r in zip(got, ref))
        assert err < 1e-12, (call, err)


def test_noalloc_inverse_rejects_oversized_and_singular_input():
    from paper_2210_02690_gb300 import load_library

    lib = load_library()
    a = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.empty_like(a)
    assert _call(lib, 257, a, out) == 1
    assert b"257" in lib.stg_last_error(None)
    assert _call(lib, 4, a, out) == 4
    eye = torch.eye(4, dtype=torch.float64, device="cuda").reshape(1, 4, 4) * 2.0
    assert _call(lib, 4, eye, out) == 0
    assert torch.allclose(out, eye / 4.0)


def test_noalloc_inverse_reports_lowest_singular_index():
    """Two singular matrices (a zero column stays exactly zero under elimination, so its pivot is
    exactly zero), both in the second launch: the message names the lower index, their outputs are
    zero and every other matrix is still inverted."""
    from paper_2210_02690_gb300 import load_library

    lib = load_library()
    n = 64
    slots = SCRATCH_DOUBLES // (n * n)
    count = slots + 50
    rng = np.random.default_rng(7)
    a_h = _well_conditioned(rng, count, n)
    lo, hi = slots + 3, slots + 41
    for i in (lo, hi):
        a_h[i, :, 5] = 0.0
    a = torch.from_numpy(a_h).cuda()
    out = torch.full_like(a, float("nan"))
    assert _call(lib, n, a, out) == 4
    assert f"matrix {lo} ".encode() in lib.stg_last_error(None)
    got = out.cpu().numpy()
    assert not np.any(got[lo]) and not np.any(got[hi])
    ok = [i for i in range(count) if i not in (lo, hi)]
    assert max(_rel(got[i], np.linalg.inv(a_h[i])) for i in ok[::17]) < 1e-12
