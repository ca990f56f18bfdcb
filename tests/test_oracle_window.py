"""The window construction behind the full-size sampled parity checks: on a mesh small enough
for the global oracle, the window's patch matrix and the rows of J x at the patch's degrees of
freedom equal those of the global Jacobian, for interior, wall, inflow, outflow and corner cells."""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, mesh
from window import window

OUT2 = si.FACE_XLO | si.FACE_YLO | si.FACE_YHI


@pytest.mark.parametrize("k", [1, 2])
def test_window_reproduces_global_patch_rows(k):
    spec = si.MeshSpec(2, (7, 5), (0.0, 0.0), (2.2, 0.41), 1, OUT2)
    w = si.channel_w(spec, k, seed=4)
    lev = mesh.Level(spec, 0, k)
    Jg = assemble.jacobian(lev, w, 1e-3, 0.005, newton=True)
    x = si.random_vector(lev.N, 9)
    y = Jg @ x
    for cx, cy in [(3, 2), (0, 2), (6, 0), (2, 4), (6, 4), (0, 0), (1, 1)]:
        _, J, gidx, dofs = window(spec, k, w, cx, cy, nu=1e-3, tau=0.005)
        gd = gidx[dofs]
        assert np.array_equal(np.sort(gd), np.sort(lev.dof[cy * 7 + cx]))
        assert np.allclose(J[np.ix_(dofs, dofs)], Jg[gd][:, gd].toarray(), rtol=0, atol=1e-13)
        assert np.allclose(J[dofs] @ x[gidx], y[gd], rtol=0, atol=1e-12)


def test_window_reproduces_global_patch_rows_3d():
    spec = si.MeshSpec(3, (4, 3, 3), (0.0, 0.0, 0.0), (1.0, 0.75, 0.75), 1, si.ALL3 & ~si.FACE_XHI)
    k = 1
    w = si.fourier_w(spec, k, seed=4)
    lev = mesh.Level(spec, 0, k)
    Jg = assemble.jacobian(lev, w, 1e-3, 0.01, newton=True)
    x = si.random_vector(lev.N, 9)
    y = Jg @ x
    for c in [(1, 1, 1), (0, 1, 2), (3, 2, 0), (3, 0, 2), (2, 2, 2), (0, 0, 0)]:
        _, J, gidx, dofs = window(spec, k, w, *c, nu=1e-3, tau=0.01)
        gd = gidx[dofs]
        cell = c[0] + 4 * (c[1] + 3 * c[2])
        assert np.array_equal(np.sort(gd), np.sort(lev.dof[cell]))
        assert np.allclose(J[np.ix_(dofs, dofs)], Jg[gd][:, gd].toarray(), rtol=0, atol=1e-13)
        assert np.allclose(J[dofs] @ x[gidx], y[gd], rtol=0, atol=1e-12)
