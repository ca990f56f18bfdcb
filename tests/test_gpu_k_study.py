"""Robustness of the GMRES-GMG solver in the time degree k in 3D (Sec. 4 runs dG(0..2) with
Q2/P1disc in 3D, Table 3.2): on the unit cube (4^3 -> 2^3, Oseen at seeded divergence-free w), the
FP64 and FP32 forms need the oracle's FGMRES iteration count within one for k = 0, 1, 2, and the
count grows by at most two from k = 0 to k = 2."""
import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC = si.MeshSpec(3, (4, 4, 4), (0.0,) * 3, (1.0,) * 3, 2, si.ALL3 & ~si.FACE_XHI)
NU, TAU = 1e-3, 0.01


def test_iteration_counts_hold_over_k_in_3d():
    import oracle
    from oracle import fgmres
    from paper_2210_02690_gb300 import Solver
    counts = {}
    for k in (0, 1, 2):
        w = si.fourier_w(SPEC, k)
        ref = oracle.Hierarchy(SPEC, k, NU, TAU, w, newton=False, nu1=2, nu2=2)
        b = ref.apply(si.reference_solution(SPEC, k))
        _, its_ref, _, ok_ref = fgmres.fgmres(ref.apply, ref.vcycle, b, rtol=1e-8)
        assert ok_ref
        for form in (dict(), dict(vcycle_prec="f32", factor_prec="f32")):
            s = Solver(SPEC, k, NU, TAU, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, linearisation="oseen",
                       **form)
            x, its, rel, ok = s.gmres_solve(torch.from_numpy(b).cuda())
            assert ok and abs(its - its_ref) <= 1, (k, form, its, its_ref)
            assert np.linalg.norm(b - ref.apply(x.cpu().numpy())) / np.linalg.norm(b) <= 1.01e-8
            s.close()
        counts[k] = its_ref
    assert counts[2] <= counts[0] + 2, counts
