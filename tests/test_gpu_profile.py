"""Instrumentation and launch overlap on the GPU.

* stg_profile brackets the finest level's colour launches of one sweep per V-cycle: one V-cycle
  records 2^d launches covering every finest patch once, and an FGMRES solve records 2^d per
  iteration.
* overlap_launches (programmatic dependent launch of the V-cycle's kernels) leaves every result
  bit-identical: each overlapped kernel waits for its predecessor before touching memory.
"""
import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (32, 16), (0.0, 0.0), (2.2, 0.41), 3, OUT2)
K, NU, TAU = 1, 1e-3, 0.01


def _solver(**opt):
    from paper_2210_02690_gb300 import Solver
    w = si.channel_w(SPEC, K)
    return Solver(SPEC, K, NU, TAU, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, **opt)


@pytest.mark.parametrize("form", [dict(), dict(vcycle_prec="f32", factor_prec="f32")])
def test_profile_samples_one_sweep_per_vcycle(form):
    s = _solver(**form)
    b = s.apply_jacobian(torch.from_numpy(si.reference_solution(SPEC, K, seed=4)).cuda())
    s.profile(True)
    s.vcycle(b)
    torch.cuda.synchronize()
    ms, launches, patches = s.profile_read()
    assert launches == 4 and patches == SPEC.n[0] * SPEC.n[1] and ms > 0.0
    s.profile(True)  # restart
    _, its, _, ok = s.gmres_solve(b)
    ms, launches, patches = s.profile_read()
    assert ok and launches == 4 * its and patches == its * SPEC.n[0] * SPEC.n[1]
    s.profile(False)
    s.close()


@pytest.mark.parametrize("form", [dict(), dict(vcycle_prec="f32", factor_prec="f32"),
                                  dict(vcycle_prec="f32", factor_prec="bf16")])
def test_overlap_launches_is_bit_identical(form):
    a, c = _solver(overlap_launches=1, **form), _solver(overlap_launches=0, **form)
    b = a.apply_jacobian(torch.from_numpy(si.reference_solution(SPEC, K, seed=5)).cuda())
    for use in (a, c):
        use.autotune()
    c.set_colour_variants(a.colour_variants())
    va, vc = a.vcycle(b), c.vcycle(b)
    assert torch.equal(va, vc)
    xa, ia, _, _ = a.gmres_solve(b)
    xc, ic, _, _ = c.gmres_solve(b)
    assert ia == ic and torch.equal(xa, xc)
    a.close()
    c.close()
