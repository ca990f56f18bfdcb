"""Host check of the closed-form row start that the FP32 Kronecker residual uses instead of
loading the block-CSR row pointer: for the structured 2D Q2 pattern (a node couples to the nodes
within its neighbouring cells: 5 per direction at interior vertex indices, 3 elsewhere), the
slots before node (ix, iy) are P(iy) S_x + w(iy) P(ix).  The reference is the pattern built the
way the library's set-up builds it, node by node."""
import pytest


def _width(i, nn):
    q = i % 2
    lo, hi = (i - 2, i + 2) if q == 0 else (i - 1, i + 1)
    return min(hi, nn - 1) - max(lo, 0) + 1


def _prefix(i):
    return 3 * i + 2 * max(0, (i + 1) // 2 - 1)


@pytest.mark.parametrize("n", [(1, 1), (2, 1), (3, 2), (4, 4), (11, 6), (88, 16), (17, 33)])
def test_closed_form_row_start_matches_the_pattern(n):
    nx, ny = 2 * n[0] + 1, 2 * n[1] + 1
    start = 0
    for iy in range(ny):
        for ix in range(nx):
            closed = _prefix(iy) * (_prefix(nx - 1) + 3) + _width(iy, ny) * _prefix(ix)
            assert closed == start, (ix, iy)
            start += _width(ix, nx) * _width(iy, ny)
