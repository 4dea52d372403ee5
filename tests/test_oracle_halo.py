"""The halo of a panel-sharded ghost fill, fixed from the oracle's literal ghost iteration
(section 3.3.1: ten Jacobi sweeps of neighbour-panel stencils that include the neighbours'
own ghost cells; no GPU).

A rank that owns one panel and fills that panel's ghost ring itself needs, from each of
the four panels that share an edge with it, the band of cells within 2H = k - 1 cells of
any of that panel's four edges, and nothing from the opposite panel.  The band is along
all edges, not only the shared one: every sweep passes dependence about H cells along the
neighbours' other edges (a neighbour's ghost value comes from its own neighbour's stencil,
which contains ghosts that come back from the first one).  Checked exactly (bitwise) by
zeroing everything outside the band, and minimality by a band one cell shallower.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _band(N, depth):
    i = np.arange(N)
    d1 = np.minimum(i, N - 1 - i)
    return np.minimum(d1[:, None], d1[None, :]) < depth  # [j][i]


@pytest.mark.parametrize("k,N", [(3, 20), (5, 24)])
def test_ghost_ring_depends_on_the_neighbours_edge_bands_of_depth_k_minus_1(k, N):
    H = (k - 1) // 2
    o = O.Oracle(N, k)
    me = (k + 1) // 2
    nbr = o.edge_tables()["B"].reshape(6, 4, N, me)[:, :, 0, 0]
    q = o.rossby_haurwitz() * (1 + 0.01 * np.random.default_rng(1).uniform(-1, 1, (6, N, N)))[None]
    full, _ = o.fill_ghosts(q)
    ring = np.ones((N + 2 * H, N + 2 * H), bool)
    ring[H:-H, H:-H] = False
    for p in range(6):
        adj = set(int(r) for r in nbr[p])
        assert len(adj) == 4 and p not in adj
        for depth, exact in ((2 * H, True), (2 * H - 1, False)):
            keep = np.zeros((6, N, N), bool)
            keep[p] = True
            for r in adj:
                keep[r] = _band(N, depth)
            ext, _ = o.fill_ghosts(np.where(keep[None], q, 0.0))
            same = np.array_equal(ext[:, p][:, ring], full[:, p][:, ring])
            assert same == exact, (p, depth)
