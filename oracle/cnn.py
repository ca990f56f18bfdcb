"""Small convolutional network for the Newton warm start (oracle; test infrastructure only).

The paper has no learned component; this is the reference for the GPU
network that predicts the next slab's end-velocity increment.  Layout: NCHW
float arrays on the Q2 node grid (H = ny-nodes, W = nx-nodes).  Layers:
3x3 convolutions with zero padding ("same" size), bias, tanh after every layer
but the last.  Loss: mean squared error over all outputs.  Written as plain
loops over the nine stencil offsets so that it can be read against the
definitions; forward and backward use float64.
"""
from __future__ import annotations

import numpy as np


def init_params(channels, seed: int = 0):
    """Weights ~ N(0, 1/(9 c_in)), zero biases, for layer sizes channels = [c0, c1, ..., cL]."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        w = rng.standard_normal((cout, cin, 3, 3)) / np.sqrt(9.0 * cin)
        params.append((w, np.zeros(cout)))
    return params


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n,o,i,j] = b[o] + sum_{c,dy,dx} w[o,c,dy,dx] x[n,c,i+dy-1,j+dx-1] (zero outside)."""
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((n, w.shape[0], h, wd)) + b[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,ncij->noij", w[:, :, dy, dx], xp[:, :, dy:dy + h, dx:dx + wd])
    return y


def forward(params, x):
    """Returns the output and the per-layer inputs/activations needed by backward."""
    acts = [x]
    for li, (w, b) in enumerate(params):
        z = conv3x3(acts[-1], w, b)
        acts.append(np.tanh(z) if li < len(params) - 1 else z)
    return acts[-1], acts


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(np.mean((y - t) ** 2))


def gradients(params, x, t):
    """(loss, [(dL/dw, dL/db) per layer]) by backpropagation."""
    y, acts = forward(params, x)
    g = 2.0 * (y - t) / y.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        if li < len(params) - 1:
            g = g * (1.0 - acts[li + 1] ** 2)          # through tanh
        xin = acts[li]
        n, c, h, wd = xin.shape
        xp = np.zeros((n, c, h + 2, wd + 2))
        xp[:, :, 1:-1, 1:-1] = xin
        gw = np.zeros_like(w)
        for dy in range(3):
            for dx in range(3):
                gw[:, :, dy, dx] = np.einsum("noij,ncij->oc", g, xp[:, :, dy:dy + h, dx:dx + wd])
        gb = g.sum(axis=(0, 2, 3))
        # input gradient: gin[n,c,i,j] = sum_{o,dy,dx} w[o,c,dy,dx] g[n,o,i-dy+1,j-dx+1]
        gp = np.zeros((n, w.shape[0], h + 2, wd + 2))
        gp[:, :, 1:-1, 1:-1] = g
        gin = np.zeros_like(xin)
        for dy in range(3):
            for dx in range(3):
                gin += np.einsum("oc,noij->ncij", w[:, :, dy, dx], gp[:, :, 2 - dy:2 - dy + h, 2 - dx:2 - dx + wd])
        grads[li] = (gw, gb)
        g = gin
    return float(np.mean((y - t) ** 2)), grads


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) of flat arrays; step counts from 1.
    Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def flatten(params):
    """Flat parameter vector: per layer w[c_out][c_in][3][3] then b[c_out]."""
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in params])


def unflatten(flat, channels):
    out, pos = [], 0
    for cin, cout in zip(channels[:-1], channels[1:]):
        nw = cout * cin * 9
        out.append((flat[pos:pos + nw].reshape(cout, cin, 3, 3).copy(), flat[pos + nw:pos + nw + cout].copy()))
        pos += nw + cout
    return out


# ---------------------------------------------------------------- warm start of the next slab
# A slab vector X (C-ABI order) holds, per Radau node a, the nodal velocities (node-major,
# component fastest; nodes x fastest) and then the P1disc coefficients per cell.  The
# network sees the Q2 node grid of a 2D mesh as an image of H = 2 n_y + 1 rows and
# W = 2 n_x + 1 columns.

def _end_vel(lev, X):
    k, R = lev.k, lev.R
    blk = k * (lev.R + lev.S)
    return np.asarray(X[blk:blk + R]).reshape(lev.nn[1], lev.nn[0], lev.dim)


def _end_pres(lev, X):
    k = lev.k
    blk = k * (lev.R + lev.S) + lev.R
    return np.asarray(X[blk:blk + lev.S])


def features(lev, X_n, X_nm1, scale_v, scale_d):
    """Network input (2d, H, W): [v_n(t_n) / scale_v, (v_n(t_n) - v_{n-1}(t_{n-1})) / scale_d]."""
    v = _end_vel(lev, X_n)
    dv = v - _end_vel(lev, X_nm1)
    return np.concatenate([np.moveaxis(v, 2, 0) / scale_v, np.moveaxis(dv, 2, 0) / scale_d])


def target(lev, X_n, X_nm1, X_np1, scale_d):
    """Training target (d(k+1), H, W), channel a*d + comp: the part of the next slab's velocity
    at Radau node a that linear extrapolation v_n + c_a dv misses, divided by scale_d."""
    from .timebasis import radau_nodes
    c = radau_nodes(lev.k)
    v = _end_vel(lev, X_n)
    dv = v - _end_vel(lev, X_nm1)
    vn1 = np.asarray(X_np1).reshape(lev.k + 1, lev.R + lev.S)[:, :lev.R].reshape(lev.k + 1, lev.nn[1], lev.nn[0],
                                                                                   lev.dim)
    out = [np.moveaxis(vn1[a] - v - c[a] * dv, 2, 0) / scale_d for a in range(lev.k + 1)]
    return np.concatenate(out)


def dirichlet_node_mask(lev):
    """(H, W) booleans: Q2 nodes on a face with Dirichlet data (bit 1 << (2 dir + side))."""
    H, W = lev.nn[1], lev.nn[0]
    m = np.zeros((H, W), dtype=bool)
    bits = lev.spec.dirichlet
    if bits & 1:
        m[:, 0] = True
    if bits & 2:
        m[:, -1] = True
    if bits & 4:
        m[0, :] = True
    if bits & 8:
        m[-1, :] = True
    return m


def guess(lev, params, X_n, X_nm1, scale_v, scale_d):
    """Initial guess for the next slab: velocity v_n + c_a dv + scale_d * net_a (net = None: 0),
    pressure p_n + c_a (p_n - p_{n-1}) (linear extrapolation).  The network term is left out
    at nodes on Dirichlet faces: the boundary data does not change, and the Nitsche penalty
    weights a boundary error with gamma / h, far above the weight of an interior error."""
    from .timebasis import radau_nodes
    c = radau_nodes(lev.k)
    d = lev.dim
    v = _end_vel(lev, X_n)
    dv = v - _end_vel(lev, X_nm1)
    p = _end_pres(lev, X_n)
    dp = p - _end_pres(lev, X_nm1)
    if params is not None:
        y, _ = forward(params, features(lev, X_n, X_nm1, scale_v, scale_d)[None])
        y = np.where(dirichlet_node_mask(lev)[None], 0.0, y[0])
    X0 = np.zeros((lev.k + 1, lev.R + lev.S))
    for a in range(lev.k + 1):
        va = v + c[a] * dv
        if params is not None:
            va = va + scale_d * np.moveaxis(y[a * d:(a + 1) * d], 0, 2)
        X0[a, :lev.R] = va.ravel()
        X0[a, lev.R:] = p + c[a] * dp
    return X0.ravel()
