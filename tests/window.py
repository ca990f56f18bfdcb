"""Window meshes for sampled full-size parity checks (test helper).

The element matrices of a cell depend only on its geometry, on w at its nodes and on which of
its faces carry Dirichlet data.  The mesh of the (up to) 3x3 cells around cell (cx, cy), with
the Dirichlet flags of the real boundary on the faces it shares with it, reproduces every entry
of the rows and columns of that cell's patch."""
import numpy as np

import stg_inputs as si
from oracle import assemble, mesh


def window(spec, k, w_full, cx, cy, nu, tau, newton=True):
    """(oracle Level, dense window Jacobian, window -> global C-ABI index map, patch dofs of
    (cx, cy) in the window numbering)."""
    nx, ny = spec.n
    h = ((spec.hi[0] - spec.lo[0]) / nx, (spec.hi[1] - spec.lo[1]) / ny)
    x0, x1 = max(cx - 1, 0), min(cx + 1, nx - 1)
    y0, y1 = max(cy - 1, 0), min(cy + 1, ny - 1)
    bits = 0
    if x0 == 0:
        bits |= spec.dirichlet & si.FACE_XLO
    if x1 == nx - 1:
        bits |= spec.dirichlet & si.FACE_XHI
    if y0 == 0:
        bits |= spec.dirichlet & si.FACE_YLO
    if y1 == ny - 1:
        bits |= spec.dirichlet & si.FACE_YHI
    wspec = si.MeshSpec(2, (x1 - x0 + 1, y1 - y0 + 1), (spec.lo[0] + x0 * h[0], spec.lo[1] + y0 * h[1]),
                        (spec.lo[0] + (x1 + 1) * h[0], spec.lo[1] + (y1 + 1) * h[1]), 1, bits)
    lev = mesh.Level(wspec, 0, k)
    gnx, gny = 2 * nx + 1, 2 * ny + 1
    R, S = 2 * gnx * gny, 3 * nx * ny
    wnx, wny = lev.nn
    jy, jx = np.divmod(np.arange(wnx * wny), wnx)
    gnode = (2 * y0 + jy) * gnx + (2 * x0 + jx)
    ey, ex = np.divmod(np.arange(lev.n_cells), lev.cells[0])
    gcell = (y0 + ey) * nx + (x0 + ex)
    idx = []
    for a in range(k + 1):
        base = a * (R + S)
        idx.append(base + (gnode[:, None] * 2 + np.arange(2)[None]).ravel())
        idx.append(base + R + (gcell[:, None] * 3 + np.arange(3)[None]).ravel())
    gidx = np.concatenate(idx)
    w_win = np.asarray(w_full).reshape(k + 1, -1)[:, (gnode[:, None] * 2 + np.arange(2)[None]).ravel()]
    J = assemble.jacobian(lev, w_win, nu, tau, newton=newton).toarray()
    cell_w = (cy - y0) * lev.cells[0] + (cx - x0)
    return lev, J, gidx, lev.dof[cell_w]
