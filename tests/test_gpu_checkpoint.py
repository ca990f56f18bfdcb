"""Checkpoint/resume of the time march: a run restored from the checkpoint of slab n solves
slab n + 1 (fallback and network warm start) bit-for-bit like the run that wrote it."""
import os

import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI
SPEC = si.MeshSpec(2, (32, 8), (0.0, 0.0), (2.2, 0.41), 3, OUT2)
CH = (4, 8, 4)


def _march():
    from paper_2210_02690_gb300.march import March
    return March(SPEC, 1, 1e-3, 0.005, si.march_initial_velocity(SPEC), si.march_inflow(SPEC, 1),
                 vcycle_prec="f32", factor_prec="f32")


def test_resume_reproduces_the_next_slab(tmp_path):
    from paper_2210_02690_gb300 import Cnn
    a = _march()
    a.run(12)
    net, sv, _, _ = a.train(CH, si.cnn_init(CH), list(range(2, 11)), epochs=5, batch=4)
    path = os.path.join(tmp_path, "march.ckpt")
    a.save(path, net, sv)
    n = len(a.X) - 1
    sd = a.scale_d(n)
    g_a = a.solver.warm_start(net, a.X[n], a.X[n - 1], sv, sd)
    ref = [a.solve_slab(n, a.solver.slab_initial_guess(a.X[n])), a.solve_slab(n, g_a)]

    b = _march()
    n_b, params, sv_b = b.load(path)
    assert n_b == n and sv_b == sv and np.array_equal(params, net.get_params())
    H, W = b.solver.node_grid()
    net_b = Cnn(CH, H, W, max_batch=1)
    net_b.set_params(params)
    g_b = b.solver.warm_start(net_b, b.X[n], b.X[n - 1], sv_b, b.scale_d(n))
    assert torch.equal(g_a, g_b)
    got = [b.solve_slab(n, b.solver.slab_initial_guess(b.X[n])), b.solve_slab(n, g_b)]
    for (Xa, sa, ia, ra, oka, _), (Xb, sb, ib, rb, okb, _) in zip(ref, got):
        assert oka and okb and (sa, ia, ra) == (sb, ib, rb)
        assert torch.equal(Xa, Xb)
    for m in (a, b):
        m.close()
    net.close()
    net_b.close()


def test_checkpoint_of_another_problem_is_rejected(tmp_path):
    from paper_2210_02690_gb300.march import March
    a = _march()
    a.run(2)
    path = os.path.join(tmp_path, "march.ckpt")
    a.save(path)
    spec2 = si.MeshSpec(2, (16, 8), (0.0, 0.0), (2.2, 0.41), 2, OUT2)
    b = March(spec2, 1, 1e-3, 0.005, si.march_initial_velocity(spec2), si.march_inflow(spec2, 1))
    with pytest.raises(ValueError):
        b.load(path)
    a.close()
    b.close()
