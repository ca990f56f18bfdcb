"""The seeded synthetic inputs (stg_inputs.py) have the properties their recipe states: exact
boundary behaviour of the curl fields, the stated amplitudes, the pressure normalisation of x*,
the batch's mesh rules and the DoF counts of the discretisation (R = d prod(2 n_i + 1) velocity
and S = (d + 1) prod(n_i) pressure values per Radau node)."""
import numpy as np
import pytest

import stg_inputs as si


def _node_xyz(spec, level=None):
    level = spec.n_levels - 1 if level is None else level
    return si.node_coords(spec, level)


@pytest.mark.parametrize("dim", [2, 3])
def test_fourier_w_has_no_normal_flow_and_unit_amplitude(dim):
    """w = curl of a series of sin(m pi u) terms: the potential vanishes on the box boundary, so
    the normal component of w does too; the field is scaled to max nodal |w| = amp."""
    spec = si.MeshSpec(dim, (8, 6) if dim == 2 else (4, 4, 3), (0.0,) * dim, (1.0, 0.7, 0.5)[:dim], 1,
                       si.ALL2 if dim == 2 else si.ALL3)
    w = si.fourier_w(spec, 1, amp=0.8)
    assert w.shape == (2, spec.dim * int(np.prod([2 * c + 1 for c in spec.n])))
    assert np.array_equal(w[0], w[1])                      # constant over the Radau nodes
    wn = w[0].reshape(-1, dim)
    assert np.max(np.linalg.norm(wn, axis=1)) == pytest.approx(0.8, rel=1e-14)
    xyz = _node_xyz(spec)
    for e in range(dim):
        for bound in (spec.lo[e], spec.hi[e]):
            on = np.isclose(xyz[:, e], bound)
            assert np.max(np.abs(wn[on, e])) <= 1e-12


def test_channel_w_inflow_profile_and_perturbation_amplitude():
    cfg = si.WORKLOADS["channel704_k1"]
    spec = si.scaled(cfg["spec"], 8)                       # 88 x 16, same recipe
    w = si.channel_w(spec, 1)[0].reshape(-1, 2)
    base = si.channel_w(spec, 1, pert=0.0)[0].reshape(-1, 2)
    xyz = _node_xyz(spec)
    H = spec.hi[1] - spec.lo[1]
    y = xyz[:, 1] - spec.lo[1]
    assert np.allclose(base[:, 0], 4 * 1.5 * y * (H - y) / H ** 2, atol=1e-15)
    assert np.max(base[:, 0]) == pytest.approx(1.5, rel=1e-12)   # mid-height is a node
    pert = w - base
    assert np.max(np.linalg.norm(pert, axis=1)) == pytest.approx(0.3, rel=1e-14)
    inflow = np.isclose(xyz[:, 0], spec.lo[0])
    assert np.max(np.abs(w[inflow, 0] - base[inflow, 0])) <= 1e-12  # normal inflow = Poiseuille
    for wall in (spec.lo[1], spec.hi[1]):
        assert np.max(np.abs(w[np.isclose(xyz[:, 1], wall), 1])) <= 1e-12  # no flow through walls


@pytest.mark.parametrize("faces,zero_mean", [(si.ALL2, True), (si.FACE_XLO | si.FACE_YLO | si.FACE_YHI, False)])
def test_reference_solution_pressure_normalisation(faces, zero_mean):
    spec = si.MeshSpec(2, (6, 4), (0.0, 0.0), (1.0, 1.0), 2, faces)
    k = 2
    x = si.reference_solution(spec, k)
    _, p = si.split_blocks(x, 2, spec.n, k)
    means = p[:, :, 0].mean(axis=1)
    if zero_mean:
        assert np.max(np.abs(means)) <= 1e-15
    else:
        assert np.max(np.abs(means)) > 1e-3


def test_batch_problems_follow_the_mesh_rules():
    probs = si.batch_problems()
    assert len(probs) == 64
    for spec, k, seed in probs:
        nx, ny = spec.n
        assert nx in (32, 64, 128, 256) and ny in (32, 64, 128, 256) and k in (1, 2)
        hx, hy = (spec.hi[0] - spec.lo[0]) / nx, (spec.hi[1] - spec.lo[1]) / ny
        assert hx == pytest.approx(hy, rel=1e-14)           # square cells
        coarse = spec.cells(0)
        assert min(coarse) == 4                              # coarsened until min(n_x, n_y) = 4
        assert spec.dirichlet == si.ALL2
    assert len({s for _, _, s in probs}) == 64


def test_dof_counts_of_the_bench_channel():
    # finest 704 x 128 and coarse 88 x 16, dG(1): (k+1)(2 (2nx+1)(2ny+1) + 3 nx ny)
    assert si.n_dofs(2, (704, 128), 1) == 2 * (2 * 1409 * 257 + 3 * 704 * 128) == 1989124
    assert si.n_dofs(2, (88, 16), 1) == 31812
    spec = si.WORKLOADS["channel704_k1"]["spec"]
    per_cycle = si.smoothed_dofs_per_cycle(spec, 1, 2, 2)
    assert per_cycle == 4 * sum(si.n_dofs(2, spec.cells(l), 1) for l in (1, 2, 3)) == 10454576
