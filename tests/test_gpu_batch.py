"""Batched solves (one CUDA graph with a branch per problem) and the colour-kernel autotuner."""
import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
PROBLEMS = [
    (si.MeshSpec(2, (16, 8), (0.0, 0.0), (2.2, 0.41), 3, OUT2), 1),
    (si.MeshSpec(2, (8, 8), (0.0, 0.0), (1.0, 1.0), 2, si.ALL2), 2),
    (si.MeshSpec(2, (32, 16), (0.0, 0.0), (2.2, 0.41), 3, OUT2), 1),
    (si.MeshSpec(2, (12, 12), (0.0, 0.0), (1.0, 1.0), 2, si.ALL2), 0),
]


def _solver(spec, k, seed, **opts):
    from paper_2210_02690_gb300 import Solver
    w = si.channel_w(spec, k, seed=seed) if spec.dirichlet == OUT2 else si.fourier_w(spec, k, seed=seed)
    return Solver(spec, k, 1e-3, 0.01, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2, **opts)


def _rhs(s, spec, k, seed):
    import oracle  # noqa: F401  (only for consistent data generation below)
    xs = si.reference_solution(spec, k, seed=seed)
    return s.apply_jacobian(torch.from_numpy(xs).cuda())


@pytest.mark.parametrize("form", [dict(), dict(vcycle_prec="f32", factor_prec="f32")])
def test_batch_reproduces_individual_solves(form):
    from paper_2210_02690_gb300 import Batch
    solvers = [_solver(spec, k, 10 + i, **form) for i, (spec, k) in enumerate(PROBLEMS)]
    rhs = [_rhs(s, spec, k, 20 + i) for i, (s, (spec, k)) in enumerate(zip(solvers, PROBLEMS))]
    single = [s.gmres_solve(b) for s, b in zip(solvers, rhs)]
    batch = Batch(solvers)
    xs, its, rel, ok = batch.gmres_solve(rhs)
    assert ok
    for (x1, it1, r1, ok1), x2, it2, r2 in zip(single, xs, its, rel):
        assert ok1 and it1 == it2 and r1 == r2
        assert torch.equal(x1, x2)
    batch.close()
    for s in solvers:
        s.close()


def test_autotune_keeps_results_bit_identical():
    spec, k = PROBLEMS[2]
    for form in (dict(), dict(vcycle_prec="f32", factor_prec="f32")):
        s = _solver(spec, k, 3, **form)
        b = _rhs(s, spec, k, 4)
        v0 = s.vcycle(b).clone()
        variant, ms = s.autotune()
        assert 0 <= variant < 13 and ms > 0
        assert torch.equal(s.vcycle(b), v0)
        s.close()


def test_batch_members_match_oracle():
    """Three members of the batch (a channel at k = 1, a square at k = 2, a square at k = 0) against
    the oracle: the same FGMRES iteration count within one and the 1e-8 true residual of the
    oracle's operator."""
    import oracle
    from oracle import fgmres
    from paper_2210_02690_gb300 import Batch
    solvers = [_solver(spec, k, 10 + i) for i, (spec, k) in enumerate(PROBLEMS)]
    refs, rhs = {}, []
    for i, (s, (spec, k)) in enumerate(zip(solvers, PROBLEMS)):
        w = si.channel_w(spec, k, seed=10 + i) if spec.dirichlet == OUT2 else si.fourier_w(spec, k, seed=10 + i)
        ref = oracle.Hierarchy(spec, k, 1e-3, 0.01, w, newton=True, nu1=2, nu2=2)
        refs[i] = ref
        rhs.append(torch.from_numpy(ref.apply(si.reference_solution(spec, k, seed=20 + i))).cuda())
    batch = Batch(solvers)
    xs, its, rel, ok = batch.gmres_solve(rhs)
    assert ok
    for i in (0, 1, 3):
        ref = refs[i]
        b = rhs[i].cpu().numpy()
        x = xs[i].cpu().numpy()
        _, its_ref, _, ok_ref = fgmres.fgmres(ref.apply, ref.vcycle, b, rtol=1e-8)
        assert ok_ref and abs(its[i] - its_ref) <= 1, (i, its[i], its_ref)
        assert np.linalg.norm(b - ref.apply(x)) / np.linalg.norm(b) <= 1.01e-8
    batch.close()
    for s in solvers:
        s.close()
