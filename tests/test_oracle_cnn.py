"""Pins of the oracle's warm-start network: forward pass against scipy's 2D
correlation, backward pass against central finite differences of the loss."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, c], w[o, c], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = cnn.init_params([4, 5, 3, 2], seed=2)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    x = rng.standard_normal((2, 4, 6, 5))
    t = rng.standard_normal((2, 2, 6, 5))
    _, grads = cnn.gradients(params, x, t)
    eps = 1e-6
    for li, (w, b) in enumerate(params):
        for arr, g in ((w, grads[li][0]), (b, grads[li][1])):
            for idx in list(np.ndindex(arr.shape))[:: max(1, arr.size // 12)]:
                old = arr[idx]
                arr[idx] = old + eps
                lp = cnn.loss(params, x, t)
                arr[idx] = old - eps
                lm = cnn.loss(params, x, t)
                arr[idx] = old
                assert abs((lp - lm) / (2 * eps) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))


def test_adam_closed_forms():
    # bias correction makes the first step lr * g / (|g| + eps); a constant gradient keeps
    # m_hat = g and v_hat = g^2, so every step has that size (Kingma & Ba, Sec. 2)
    g = np.array([3.0, -0.5, 1e-3, -2.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    m = v = np.zeros(4)
    lr, eps = 0.01, 1e-8
    th = theta
    for step in (1, 2, 3):
        th, m, v = cnn.adam_step(th, g, m, v, step, lr, eps=eps)
        assert np.allclose(th, theta - step * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)


def test_flatten_round_trip():
    ch = [4, 3, 2]
    p = cnn.init_params(ch, seed=3)
    q = cnn.unflatten(cnn.flatten(p), ch)
    assert all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) for a, b in zip(p, q))
    assert cnn.flatten(p).size == 4 * 3 * 9 + 3 + 3 * 2 * 9 + 2


def _slab_from_field(lev, vel, pres, t0, tau, radau):
    """C-ABI slab vector whose velocity/pressure at Radau node a are vel(t0 + c_a tau), pres(...)."""
    X = np.zeros((lev.k + 1, lev.R + lev.S))
    for a, ca in enumerate(radau):
        X[a, :lev.R] = vel(t0 + ca * tau).ravel()
        X[a, lev.R:] = pres(t0 + ca * tau)
    return X.ravel()


def _setup(k=1):
    import stg_inputs as si
    from oracle import mesh, timebasis
    spec = si.MeshSpec(2, (6, 3), (0.0, 0.0), (2.2, 0.41), 1, si.FACE_XLO)
    lev = mesh.Level(spec, 0, k)
    xy = si.node_coords(spec, 0)
    return si, lev, xy, timebasis.radau_nodes(k)


def test_features_follow_the_node_grid():
    si, lev, xy, c = _setup()
    f = lambda x, y: np.stack([np.sin(x) + y, x * y * y], axis=-1)   # noqa: E731
    vel = lambda t: f(xy[:, 0], xy[:, 1]) * (1 + t)                   # noqa: E731
    pres = lambda t: np.full(lev.S, t)                               # noqa: E731
    Xn = _slab_from_field(lev, vel, pres, 1.0, 0.1, c)
    Xm = _slab_from_field(lev, vel, pres, 0.9, 0.1, c)
    F = cnn.features(lev, Xn, Xm, 2.0, 0.5)
    assert F.shape == (4, lev.nn[1], lev.nn[0])
    xs = np.linspace(0.0, 2.2, lev.nn[0])
    ys = np.linspace(0.0, 0.41, lev.nn[1])
    for j in (0, 3, lev.nn[1] - 1):
        for i in (0, 5, lev.nn[0] - 1):
            fv = f(xs[i], ys[j])
            assert np.allclose(F[:2, j, i], fv * 2.1 / 2.0, atol=1e-14)
            assert np.allclose(F[2:, j, i], fv * 0.1 / 0.5, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2])
def test_linear_in_time_trajectory_is_extrapolated_exactly(k):
    si, lev, xy, c = _setup(k)
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((2, lev.n_nodes, 2))
    P, Q = rng.standard_normal((2, lev.S))
    vel = lambda t: A + B * t                                         # noqa: E731
    pres = lambda t: P + Q * t                                        # noqa: E731
    tau = 0.05
    Xm, Xn, Xp = (_slab_from_field(lev, vel, pres, t0, tau, c) for t0 in (0.3 - tau, 0.3, 0.3 + tau))
    assert np.allclose(cnn.guess(lev, None, Xn, Xm, 1.0, 1.0), Xp, atol=1e-13)
    assert np.abs(cnn.target(lev, Xn, Xm, Xp, 0.7)).max() < 1e-12


def test_guess_places_network_channels_at_radau_nodes():
    si, lev, xy, c = _setup(2)
    rng = np.random.default_rng(6)
    Xn, Xm = rng.standard_normal((2, 3 * (lev.R + lev.S)))
    bias = np.arange(6, dtype=float) + 1.0          # channel a*d + comp
    params = [(np.zeros((6, 4, 3, 3)), bias)]
    base = cnn.guess(lev, None, Xn, Xm, 1.0, 0.5).reshape(3, lev.R + lev.S)
    got = cnn.guess(lev, params, Xn, Xm, 1.0, 0.5).reshape(3, lev.R + lev.S)
    on_xlo = np.isclose(xy[:, 0], 0.0)          # the only Dirichlet face of this mesh
    assert on_xlo.sum() == lev.nn[1]
    for a in range(3):
        dv = (got[a, :lev.R] - base[a, :lev.R]).reshape(-1, 2)
        assert np.allclose(dv[~on_xlo], 0.5 * bias[2 * a:2 * a + 2], atol=1e-14)
        assert np.array_equal(dv[on_xlo], np.zeros((on_xlo.sum(), 2)))
        assert np.array_equal(got[a, lev.R:], base[a, lev.R:])


def test_dirichlet_mask_marks_the_faces():
    import stg_inputs as si
    from oracle import mesh
    spec = si.MeshSpec(2, (4, 2), (0.0, 0.0), (1.0, 1.0), 1, si.FACE_XHI | si.FACE_YLO)
    lev = mesh.Level(spec, 0, 0)
    m = cnn.dirichlet_node_mask(lev)
    xy = si.node_coords(spec, 0).reshape(lev.nn[1], lev.nn[0], 2)
    assert np.array_equal(m, np.isclose(xy[..., 0], 1.0) | np.isclose(xy[..., 1], 0.0))
