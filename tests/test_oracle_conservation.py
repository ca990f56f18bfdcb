"""Cellwise mass conservation of the oracle's discrete solution (Sec. 2, Eq. (2.1)-(2.2)).

P1disc contains, on every cell K, the constant and the linear functions xi_m.  The pressure rows
of the slab problem therefore say, for each cell K, Radau node a and P1disc function xi_m,

    (div v_h(t_a), xi_m)_K - < (v_h(t_a) - g(t_a)) . n, xi_m >_{dK cap Gamma_D} = 0,

with the Dirichlet data g entering through B_GammaD on the right-hand side.  Here the two
integrals are computed directly from the solved nodal velocities and the data (basis gradients and
face rules of the element), not from the assembled blocks, so a mis-signed or missing boundary term
in the pressure rows, a wrong pressure right-hand side or a wrong face scaling breaks the identity.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import stg_inputs as si
from oracle import assemble, element, mesh, timebasis

NU, TAU, T0 = 0.05, 0.3, 0.2


def gdata(x, t):
    """Smooth Dirichlet data, not divergence-free (the net inflow is not zero)."""
    d = x.shape[1]
    out = np.stack([np.sin(1.3 * x[:, 0] + t) + x[:, 1], np.cos(0.7 * x[:, 1]) - t * x[:, 0]]
                   + ([0.4 * x[:, 2] + t * x[:, 0] * x[:, 1]] if d == 3 else []), 1)
    return out


def fdata(x, t):
    d = x.shape[1]
    return np.stack([np.cos(x[:, 1] + t)] + [x[:, 0] * (1 - t)] + ([np.sin(x[:, 0])] if d == 3 else []), 1)


def cell_balance(lev, X, g):
    """(div v_h, xi_m)_K - <(v_h - g) . n, xi_m>_{dK cap Gamma_D} for every (a, K, m)."""
    d, k = lev.dim, lev.k
    h = np.asarray(lev.h)
    cn = timebasis.radau_nodes(k)
    pts, qw = element.cell_rule(d)
    det = np.prod(h / 2.0)
    _, gref = element.q2_basis(pts)
    gphys = gref * (2.0 / h)
    pb = element.p1disc_basis(pts)
    cen = lev.cell_centres()
    out = np.zeros((k + 1, lev.n_cells, d + 1))
    for a in range(k + 1):
        ta = T0 + TAU * cn[a]
        vn = X[lev.vel_index(a, np.arange(lev.n_nodes)[:, None], np.arange(d)[None, :])]   # (nodes, d)
        vc = vn[lev.cell_nodes]                                                             # (nc, nloc, d)
        div = np.einsum("qic,kic->kq", gphys, vc)                                           # (nc, nq)
        out[a] = np.einsum("q,kq,qm->km", qw * det, div, pb)
        for e, side, cells in lev.boundary_faces():
            if not lev.is_dirichlet(e, side):
                continue
            fp, fw = element.face_rule(d, e, side)
            fqw = fw * np.prod(np.delete(h, e) / 2.0)
            fv, _ = element.q2_basis(fp)
            nrm = np.zeros(d)
            nrm[e] = 1.0 if side == 1 else -1.0
            vf = np.einsum("qi,kic->kqc", fv, vc[cells])
            xf = cen[cells][:, None, :] + fp[None] * (h / 2.0)
            gf = g(xf.reshape(-1, d), ta).reshape(len(cells), -1, d)
            flux = (vf - gf) @ nrm                                                          # (ncells, nq)
            out[a, cells] -= np.einsum("q,kq,qm->km", fqw, flux, element.p1disc_basis(fp))
    return out


@pytest.mark.parametrize("dim,k,newton", [(2, 0, False), (2, 1, True), (2, 2, False), (3, 1, True)])
def test_cellwise_mass_conservation(dim, k, newton):
    rng = np.random.default_rng(si.BASE_SEED + 10 * dim + k)
    if dim == 2:
        spec = si.MeshSpec(2, (4, 3), (0.0, 0.0), (1.0, 0.6), 1, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI)
    else:
        spec = si.MeshSpec(3, (2, 2, 2), (0.0,) * 3, (1.0, 0.8, 0.6), 1, si.ALL3 & ~si.FACE_XHI)
    lev = mesh.Level(spec, 0, k)
    w = rng.standard_normal((k + 1) * lev.n_nodes * dim)
    jac = assemble.jacobian(lev, w, NU, TAU, newton)
    v_prev = rng.standard_normal(lev.R)
    b = assemble.rhs_linear(lev, fdata, gdata, v_prev, NU, TAU, t0=T0)
    X = spla.spsolve(jac.tocsc(), b)
    assert np.linalg.norm(jac @ X - b) <= 1e-10 * np.linalg.norm(b)
    bal = cell_balance(lev, X, gdata)
    # each entry is a sum of O(1) terms; the solve leaves rounding of order 1e-13
    scale = np.abs(X).max()
    assert np.abs(bal).max() <= 1e-10 * scale, np.abs(bal).max()


def test_balance_detects_a_wrong_flux_sign():
    """The check is sensitive: the same balance with the boundary flux counted with the wrong
    sign does not vanish on the solved problem (the Dirichlet data carry net flux)."""
    k = 1
    spec = si.MeshSpec(2, (4, 3), (0.0, 0.0), (1.0, 0.6), 1, si.FACE_XLO | si.FACE_YLO | si.FACE_YHI)
    lev = mesh.Level(spec, 0, k)
    rng = np.random.default_rng(si.BASE_SEED)
    w = rng.standard_normal((k + 1) * lev.n_nodes * 2)
    jac = assemble.jacobian(lev, w, NU, TAU, False)
    b = assemble.rhs_linear(lev, fdata, gdata, None, NU, TAU, t0=T0)
    X = spla.spsolve(jac.tocsc(), b)
    good = cell_balance(lev, X, gdata)
    flipped = cell_balance(lev, X, lambda x, t: -gdata(x, t))
    assert np.abs(good).max() <= 1e-10 * np.abs(X).max()
    assert np.abs(flipped).max() > 1e-3
