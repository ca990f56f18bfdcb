"""Window meshes for sampled full-size parity checks (test helper).

The element matrices of a cell depend only on its geometry, on w at its nodes and on which of
its faces carry Dirichlet data.  The mesh of the (up to) 3^d cells around a cell, with the
Dirichlet flags of the real boundary on the faces it shares with it, reproduces every entry
of the rows and columns of that cell's patch.  Works in 2D and 3D."""
import numpy as np

import stg_inputs as si
from oracle import assemble, mesh


def window(spec, k, w_full, *cell, nu, tau, newton=True):
    """(oracle Level, dense window Jacobian, window -> global C-ABI index map, patch dofs of the
    cell with multi-index `cell` in the window numbering)."""
    d = spec.dim
    n = spec.n
    h = [(spec.hi[e] - spec.lo[e]) / n[e] for e in range(d)]
    lo_c = [max(cell[e] - 1, 0) for e in range(d)]
    hi_c = [min(cell[e] + 1, n[e] - 1) for e in range(d)]
    bits = 0
    for e in range(d):
        if lo_c[e] == 0:
            bits |= spec.dirichlet & (1 << (2 * e))
        if hi_c[e] == n[e] - 1:
            bits |= spec.dirichlet & (1 << (2 * e + 1))
    wspec = si.MeshSpec(d, tuple(hi_c[e] - lo_c[e] + 1 for e in range(d)),
                        tuple(spec.lo[e] + lo_c[e] * h[e] for e in range(d)),
                        tuple(spec.lo[e] + (hi_c[e] + 1) * h[e] for e in range(d)), 1, bits)
    lev = mesh.Level(wspec, 0, k)
    gnn = [2 * n[e] + 1 for e in range(d)]
    R, S = d * int(np.prod(gnn)), (d + 1) * int(np.prod(n))
    # window node / cell multi-indices (x fastest) -> global numbers
    wn = np.stack([g.ravel(order="F") for g in np.meshgrid(*[np.arange(m) for m in lev.nn], indexing="ij")],
                  axis=1)
    wc = np.stack([g.ravel(order="F") for g in np.meshgrid(*[np.arange(m) for m in lev.cells], indexing="ij")],
                  axis=1)
    gnode = np.zeros(len(wn), dtype=np.int64)
    gcell = np.zeros(len(wc), dtype=np.int64)
    sn = sc = 1
    for e in range(d):
        gnode += (2 * lo_c[e] + wn[:, e]) * sn
        gcell += (lo_c[e] + wc[:, e]) * sc
        sn *= gnn[e]
        sc *= n[e]
    idx = []
    for a in range(k + 1):
        base = a * (R + S)
        idx.append(base + (gnode[:, None] * d + np.arange(d)[None]).ravel())
        idx.append(base + R + (gcell[:, None] * (d + 1) + np.arange(d + 1)[None]).ravel())
    gidx = np.concatenate(idx)
    w_win = np.asarray(w_full).reshape(k + 1, -1)[:, (gnode[:, None] * d + np.arange(d)[None]).ravel()]
    J = assemble.jacobian(lev, w_win, nu, tau, newton=newton).toarray()
    cw = 0
    s = 1
    for e in range(d):
        cw += (cell[e] - lo_c[e]) * s
        s *= lev.cells[e]
    return lev, J, gidx, lev.dof[cw]
