"""Variable slab length tau_n (Sec. 4 marches with tau = 0.1, 0.05, 0.01): stg_set_slab_length
re-assembles every level of a live context; operators, V-cycles and Newton slabs then match the
oracle built with the new tau, over a march whose slab length changes from slab to slab."""
import numpy as np
import pytest

import stg_inputs as si
from oracle import mesh, newton

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (16, 8), (0.0, 0.0), (2.2, 0.41), 3, OUT2)
K, NU = 1, 1e-3


def test_set_slab_length_matches_fresh_oracle():
    from paper_2210_02690_gb300 import Solver
    import oracle
    w = si.channel_w(SPEC, K)
    gpu = Solver(SPEC, K, NU, 0.02, torch.from_numpy(w.ravel()).cuda(), nu1=2, nu2=2)
    for tau in (0.005, 0.1):
        gpu.set_slab_length(tau)
        ref = oracle.Hierarchy(SPEC, K, NU, tau, w, newton=True, nu1=2, nu2=2)
        x = si.random_vector(ref.fine.N, 3)
        y = gpu.apply_jacobian(torch.from_numpy(x).cuda()).cpu().numpy()
        y_ref = ref.apply(x)
        assert np.linalg.norm(y - y_ref) < 64 * np.finfo(float).eps * np.linalg.norm(abs(ref.J[-1]) @ np.abs(x))
        b = ref.apply(si.reference_solution(SPEC, K, seed=9))
        v = gpu.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
        v_ref = ref.vcycle(b)
        assert np.linalg.norm(v - v_ref) / np.linalg.norm(v_ref) < 1e-12
    gpu.close()


def test_march_with_changing_slab_length():
    from paper_2210_02690_gb300 import Solver
    lev = mesh.Level(SPEC, SPEC.n_levels - 1, K)
    v0 = si.channel_w(SPEC, 0, pert=0.3)[0]
    g = np.repeat(si.channel_w(SPEC, 0, pert=0.0)[0][None], K + 1, axis=0)
    X0 = np.concatenate([np.concatenate([v0, np.zeros(lev.S)])] * (K + 1))
    taus = [0.02, 0.01, 0.005, 0.01]
    solver = Solver(SPEC, K, NU, taus[0], torch.from_numpy(np.concatenate([v0] * (K + 1))).cuda(), nu1=2, nu2=2,
                    gmres_rtol=1e-12)
    Xo, vprev = X0.copy(), v0.copy()
    Xg, vg, gg = torch.from_numpy(X0).cuda(), torch.from_numpy(v0).cuda(), torch.from_numpy(g.ravel()).cuda()
    for tau in taus:
        solver.set_slab_length(tau)
        b = newton.rhs_nodal(lev, None, g, vprev, NU, tau)
        Xo, steps_ref, _, _ = newton.newton_slab(SPEC, K, NU, tau, Xo, b, rtol=1e-10, gmres_rtol=1e-12)
        Xg, steps, _, _, ok = solver.newton_slab(Xg, v_prev=vg, g=gg, rtol=1e-10)
        assert ok and steps == steps_ref
        assert np.linalg.norm(Xg.cpu().numpy() - Xo) / np.linalg.norm(Xo) < 1e-9
        vprev = newton.end_value(lev, Xo)
        Xo = np.concatenate([Xo.reshape(K + 1, -1)[-1]] * (K + 1))
        vg = Xg[K * (lev.R + lev.S):K * (lev.R + lev.S) + lev.R].clone()
        Xg = solver.slab_initial_guess(Xg)
    solver.close()
