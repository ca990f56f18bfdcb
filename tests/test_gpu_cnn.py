"""Parity of the warm-start network kernels (through the C ABI) with the oracle.

Tolerances: the GPU computes in FP32 (unit roundoff u = 6e-8).  Each output of a
layer is a dot product of length 9 c_in <= 144 and each weight gradient a sum of
~200 pixels per tile (FP32) followed by an FP64 sum over tiles, so the worst-case
relative rounding of one layer is below 300 u = 2e-5; with three layers stacked,
norm-wise agreement to 1e-4 is a bound with margin.  Adam is elementwise
(a few roundings per entry): 1e-6 relative to the parameters.  The packing
kernels round FP64 values to FP32 once (1e-7) and the guess is FP64 arithmetic
(exact formula: 1e-15; with the FP32 network term: 1e-6 of that term).
"""
import numpy as np
import pytest

import stg_inputs as si
from oracle import cnn as ocnn
from oracle import mesh as omesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(np.asarray(b, float)),
                                                                           1e-300)


def _net(channels, H, W, B, seed):
    from paper_2210_02690_gb300 import Cnn
    flat = si.cnn_init(channels, seed=seed, last_scale=1.0)
    rng = np.random.default_rng(seed + 1)
    # non-zero biases so that every term of the oracle's formulas is exercised
    params = ocnn.unflatten(flat.astype(np.float64), channels)
    params = [(w, 0.1 * rng.standard_normal(b.shape)) for w, b in params]
    flat = ocnn.flatten(params).astype(np.float32)
    params = ocnn.unflatten(flat.astype(np.float64), channels)
    net = Cnn(channels, H, W, max_batch=B)
    net.set_params(flat)
    return net, params


SHAPES = [((4, 16, 16, 4), 13, 70, 3),     # two column tiles, ragged row tile
          ((3, 5, 2), 7, 9, 2),            # channel pairs fewer than the threads of a tile
          ((2, 32, 1), 5, 130, 1),         # widest layer, three column tiles
          ((4, 16, 16, 4), 65, 257, 2)]    # the march's node grid (128 x 32 cells)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}-{s[1]}x{s[2]}")
def test_forward_and_gradients_match_oracle(shape):
    channels, H, W, B = shape
    net, params = _net(channels, H, W, B, seed=H * 1000 + W)
    rng = np.random.default_rng(W)
    x = rng.standard_normal((B, channels[0], H, W)).astype(np.float32)
    t = rng.standard_normal((B, channels[-1], H, W)).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref, _ = ocnn.forward(params, x.astype(np.float64))
    assert rel(y, y_ref) < 1e-4
    loss, g = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    loss_ref, grads_ref = ocnn.gradients(params, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - loss_ref) < 1e-5 * loss_ref
    g_ref = ocnn.flatten(grads_ref)
    g = g.cpu().numpy()
    pos = 0
    for li, (gw, gb) in enumerate(grads_ref):
        nw, nb = gw.size, gb.size
        assert rel(g[pos:pos + nw], gw.ravel()) < 1e-4, ("weights", li)
        assert rel(g[pos + nw:pos + nw + nb], gb) < 1e-4, ("bias", li)
        pos += nw + nb
    assert np.abs(g - g_ref).max() < 1e-4 * np.abs(g_ref).max()
    net.close()


def test_adam_matches_oracle():
    channels = (3, 4, 2)
    net, params = _net(channels, 5, 6, 1, seed=3)
    theta = ocnn.flatten(params)
    rng = np.random.default_rng(4)
    m = v = np.zeros_like(theta)
    for step in (1, 2, 3):
        g = rng.standard_normal(theta.size) * 10.0 ** rng.integers(-4, 1, theta.size)
        net.adam_step(torch.from_numpy(g.astype(np.float32)).cuda(), 1e-2)
        theta, m, v = ocnn.adam_step(theta, g.astype(np.float32).astype(np.float64), m, v, step, 1e-2)
        assert rel(net.get_params(), theta) < 1e-6
    net.close()


def test_training_is_deterministic_and_learns():
    from paper_2210_02690_gb300 import Cnn
    channels = (4, 8, 4)
    H, W, S = 17, 33, 24
    rng = np.random.default_rng(8)
    x = rng.standard_normal((S, 4, H, W)).astype(np.float32)
    # a target the network can represent: a fixed 3x3 filter of the input
    p_true = ocnn.unflatten(si.cnn_init((4, 4), seed=9, last_scale=1.0).astype(np.float64), (4, 4))
    t, _ = ocnn.forward(p_true, x.astype(np.float64))
    order = np.concatenate([np.random.default_rng(e).permutation(S) for e in range(40)])
    p0 = si.cnn_init(channels, seed=10)
    runs = []
    for _ in range(2):
        net = Cnn(channels, H, W, max_batch=8)
        net.set_params(p0)
        losses = net.train(torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda(), order, 8,
                           3e-3)
        runs.append((net.get_params(), losses))
        net.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    losses = runs[0][1]
    assert losses[-10:].mean() < 0.2 * losses[:3].mean()


def test_train_rejects_bad_indices():
    from paper_2210_02690_gb300 import Cnn, StgError
    net = Cnn((2, 2), 4, 4, max_batch=2)
    x = torch.zeros((3, 2, 4, 4), device="cuda")
    with pytest.raises(StgError):
        net.train(x, x, np.array([0, 3]), 2, 1e-3)
    net.close()


OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI


@pytest.mark.parametrize("k", [1, 2])
def test_warm_start_packing_matches_oracle(k):
    from paper_2210_02690_gb300 import Solver
    spec = si.MeshSpec(2, (16, 8), (0.0, 0.0), (2.2, 0.41), 2, OUT2)
    w = si.channel_w(spec, k)
    s = Solver(spec, k, 1e-3, 0.005, torch.from_numpy(w.ravel()).cuda())
    lev = omesh.Level(spec, spec.n_levels - 1, k)
    rng = np.random.default_rng(k)
    Xm, Xn, Xp = rng.standard_normal((3, lev.N))
    d = lambda a: torch.from_numpy(a).cuda()                        # noqa: E731
    sv, sd = 1.3, 0.02
    f = s.warm_features(d(Xn), d(Xm), sv, sd).cpu().numpy()
    assert rel(f, ocnn.features(lev, Xn, Xm, sv, sd)) < 1e-7
    t = s.warm_target(d(Xn), d(Xm), d(Xp), sd).cpu().numpy()
    assert rel(t, ocnn.target(lev, Xn, Xm, Xp, sd)) < 1e-7
    g0 = s.warm_start(None, d(Xn), d(Xm), sv, sd).cpu().numpy()
    ref0 = ocnn.guess(lev, None, Xn, Xm, sv, sd)
    assert rel(g0, ref0) < 1e-15
    from paper_2210_02690_gb300 import Cnn
    channels = (4, 8, 2 * (k + 1))
    net = Cnn(channels, 2 * 8 + 1, 2 * 16 + 1, max_batch=1)
    flat = si.cnn_init(channels, seed=11, last_scale=1.0)
    net.set_params(flat)
    params = ocnn.unflatten(flat.astype(np.float64), channels)
    g1 = s.warm_start(net, d(Xn), d(Xm), sv, sd).cpu().numpy()
    ref1 = ocnn.guess(lev, params, Xn, Xm, sv, sd)
    assert rel(g1 - g0, ref1 - ref0) < 1e-5
    a, b = s.warm_scales(d(Xn), d(Xm))
    vn = Xn.reshape(k + 1, -1)[k, :lev.R]
    vm = Xm.reshape(k + 1, -1)[k, :lev.R]
    assert abs(a - np.sqrt(np.mean(vn ** 2))) < 1e-13 and abs(b - np.sqrt(np.mean((vn - vm) ** 2))) < 1e-13
    bad = Cnn((4, 2 * (k + 1)), 17, 35, max_batch=1)   # wrong grid width
    from paper_2210_02690_gb300 import StgError
    with pytest.raises(StgError):
        s.warm_start(bad, d(Xn), d(Xm), sv, sd)
    bad.close()
    net.close()
    s.close()
