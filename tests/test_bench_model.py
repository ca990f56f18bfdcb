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


def test_every_colour_variant_has_a_kernel_name():
    """The bench names the kernel behind any of the 17 variants the autotuner may pick (warp form
    0..8, staged 9..16 with one or two rows per thread); the staged names carry the stage count
    of the shape table and the rows per thread."""
    import bench
    names = [bench.colour_kernel_name(v) for v in range(17)]
    assert all("vanka_colour" in n for n in names)
    assert names[11].startswith("vanka_colour_bulk_kernel<float,float,2,1>")
    assert names[15].startswith("vanka_colour_bulk_kernel<float,float,2,2>")
    assert names[10].startswith("vanka_colour_bulk_kernel<float,float,3,1>")


def test_colour_fraction_reports_the_fp64_pipe_and_measured_traffic():
    import bench
    # one full-size FP64 launch: 22 528 patches of 42 in 0.114 ms
    f = bench.colour_fraction(1, "f64", 0.114, 1, 22528, 6779.4, 11)
    flops = 2.0 * 42 * 42 * 22528
    assert abs(f["fp64"]["tflops"] - flops / 0.114e-3 / 1e12) < 1e-9
    assert f["traffic"] == bench.MEASURED_TRAFFIC_PER_PATCH[("f64", 11)] * 22528
    g = bench.colour_fraction(1, "bf16", 0.028, 1, 22528, 6779.4, 12)
    assert "traffic" not in g and "fp64" not in g
