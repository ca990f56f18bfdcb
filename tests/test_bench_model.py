"""The bench's algorithmic byte model: the number of Q2 node-pair blocks it counts equals the
block structure of the oracle's velocity operator, and a sweep's byte count adds up from its
parts with the factor and vector sizes of each precision form."""
import numpy as np
import pytest

import stg_inputs as si
from oracle import assemble, mesh


@pytest.mark.parametrize("cells", [(4, 2), (3, 5), (1, 1), (2, 2, 3)])
def test_block_couplings_match_oracle_structure(cells):
    import bench
    dim = len(cells)
    spec = si.MeshSpec(dim, cells, (0.0,) * dim, (1.0,) * dim, 1, (1 << (2 * dim)) - 1)
    lev = mesh.Level(spec, 0, 0)
    J = assemble.jacobian(lev, np.ones((1, lev.R)), 1e-3, 0.01, True).tocsr()
    coo = J[:lev.R][:, :lev.R].tocoo()
    assert len(set(zip(coo.row // dim, coo.col // dim))) == bench.q2_block_couplings(cells)


def test_sweep_bytes_parts():
    import bench
    cells, k = (704, 128), 1
    n, ncell = 42, 704 * 128
    N = si.n_dofs(2, cells, k)
    b32 = bench.sweep_bytes(2, cells, k, "f32")
    b16 = bench.sweep_bytes(2, cells, k, "bf16")
    b64 = bench.sweep_bytes(2, cells, k, "f64")
    assert b32["colour"] == ncell * (n * n * 4 + 3 * n * 4)
    assert b32["colour"] - b16["colour"] == ncell * n * n * 2
    assert b32["update"] == 16 * N and b64["update"] == 32 * N
    assert b32["total"] == b32["residual"] + b32["colour"] + b32["update"]
    # the FP32 Kronecker operator is smaller than the dense FP64 blocks
    assert b32["residual"] < b64["residual"] / 2
