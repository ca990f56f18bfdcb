"""Pins of the oracle's injection of the linearisation velocity to coarse levels (reading A9:
coarse operators are rediscretised with w taken at the coarse Q2 nodes, Sec. 3).

Two checks that do not reuse the oracle's own index arithmetic:
* geometric: the injected value at every coarse node is the fine value at the fine node with the
  same coordinates (matched by position, so a wrong stride, a transposed index or fine node g
  instead of 2g fails), bit for bit, for every Radau node and component;
* interpolation: a coarse Q2 field (random nodal values), prolongated to the fine mesh by the
  nested-space prolongation (pinned separately by its reproduction of coarse FE functions), is
  injected back to the same coarse values.
"""
import numpy as np
import pytest

import stg_inputs as si
from oracle import mesh, multigrid, transfer

SPECS = {
    "channel2d": si.MeshSpec(2, (12, 4), (0.0, 0.0), (2.2, 0.41), 3, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI),
    "rect2d_offset": si.MeshSpec(2, (4, 8), (0.3, -0.2), (1.3, 0.5), 3, si.ALL2),
    "box3d": si.MeshSpec(3, (4, 2, 6), (0.0, 0.0, 0.0), (1.0, 0.5, 1.5), 2, si.ALL3),
}


def _match(coarse_xyz, fine_xyz):
    """Index of the fine node at each coarse node's position (unique, within 1e-12)."""
    key = {tuple(np.round(p, 10)): i for i, p in enumerate(fine_xyz)}
    idx = np.array([key[tuple(np.round(p, 10))] for p in coarse_xyz])
    assert np.allclose(fine_xyz[idx], coarse_xyz, atol=1e-12, rtol=0)
    return idx


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("k", [0, 2])
def test_injection_takes_the_fine_value_at_the_same_position(name, k):
    spec = SPECS[name]
    for lf in range(spec.n_levels - 1, 0, -1):
        fine, coarse = mesh.Level(spec, lf, k), mesh.Level(spec, lf - 1, k)
        rng = np.random.default_rng(lf)
        w_f = rng.standard_normal((k + 1, fine.R))
        w_c = multigrid.inject_w(w_f, fine, coarse)
        assert w_c.shape == (k + 1, coarse.R)
        idx = _match(si.node_coords(spec, lf - 1), si.node_coords(spec, lf))
        d = spec.dim
        expect = w_f.reshape(k + 1, fine.n_nodes, d)[:, idx, :].reshape(k + 1, -1)
        assert np.array_equal(w_c, expect)


@pytest.mark.parametrize("name", list(SPECS))
def test_injection_inverts_prolongation_of_coarse_q2_fields(name):
    spec = SPECS[name]
    k = 1
    lf = spec.n_levels - 1
    fine, coarse = mesh.Level(spec, lf, k), mesh.Level(spec, lf - 1, k)
    P = transfer.prolongation(coarse, fine)
    rng = np.random.default_rng(5)
    xc = rng.standard_normal(coarse.N)
    xf = P @ xc
    vf = xf.reshape(k + 1, fine.R + fine.S)[:, :fine.R]
    vc = xc.reshape(k + 1, coarse.R + coarse.S)[:, :coarse.R]
    got = multigrid.inject_w(vf, fine, coarse)
    assert np.max(np.abs(got - vc)) < 1e-14 * np.max(np.abs(vc))


def test_injection_pin_catches_planted_mistakes():
    """The geometric check fails for the plausible mistakes: fine node g instead of 2g, swapped strides."""
    spec = SPECS["channel2d"]
    fine, coarse = mesh.Level(spec, 2, 0), mesh.Level(spec, 1, 0)
    w_f = np.random.default_rng(0).standard_normal((1, fine.R))
    idx = _match(si.node_coords(spec, 1), si.node_coords(spec, 2))
    expect = w_f.reshape(1, fine.n_nodes, 2)[:, idx, :].reshape(1, -1)
    grids = np.meshgrid(*[np.arange(n) for n in coarse.nn], indexing="ij")
    g = np.stack([gg.ravel(order="F") for gg in grids], axis=1)
    wn = w_f.reshape(1, fine.n_nodes, 2)
    wrong_g = wn[:, fine.node_number(np.minimum(g, np.asarray(fine.nn) - 1)), :].reshape(1, -1)
    gs = 2 * g[:, ::-1]
    gs = np.minimum(gs, np.asarray(fine.nn) - 1)
    wrong_stride = wn[:, fine.node_number(gs), :].reshape(1, -1)
    assert not np.array_equal(wrong_g, expect)
    assert not np.array_equal(wrong_stride, expect)
