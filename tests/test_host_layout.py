"""Host-side node coordinates from the library (dg_layout_coordinates_host) equal the oracle's LGL
grid: the library's own LGL points (long-double Newton, barycentric weights) against the
oracle's; no GPU needed."""
import numpy as np
import pytest

from oracle import dg


@pytest.mark.parametrize("n,N,lo,hi", [((3, 2, 2), 5, (-1, 0, 2), (1, 1, 3)), ((1, 1, 1), 10, (0, 0, 0), (1, 2, 3)),
                                       ((4, 1, 3), 2, (-20, -20, -20), (20, 20, 20))])
def test_host_coordinates_match_oracle_grid(n, N, lo, hi):
    import __graft_entry__

    __graft_entry__._build_module().build()
    import paper_2111_06767_gb300 as dgg

    x, y, z = dgg.host_coordinates(dgg.make_desc(lo, hi, n, N))
    X, Y, Z = dg.BoxGrid(lo, hi, n, N, 1.5).coordinates()
    for a, b in ((x, X), (y, Y), (z, Z)):
        assert np.abs(a - b.ravel()).max() <= 1e-14 * max(1.0, np.abs(b).max())
