"""Host-side logic of the input generators that the GPU paths rely on (no GPU needed):
the multi-block split behind the linked batch, and the C-grid cut nodes."""
import numpy as np

from paper_2101_05886_gb300 import inputs as I


def test_split_grid_nodes_links_and_states():
    g = I.periodic_wavy_3d((20, 12, 10), L=10.0, amp=0.08, Gn=6)
    for direction, sizes in ((0, (7, 5, 8)), (1, (6, 6)), (2, (3, 7))):
        parts, links = I.split_grid(g, direction, sizes)
        ax = 3 - direction
        a0 = 0
        for b, (p, n) in enumerate(zip(parts, sizes)):
            assert p.n[direction] == n and p.Gn == g.Gn
            sl = [slice(None)] * 4
            sl[ax] = slice(a0, a0 + n + 2 * g.Gn)     # the part's ghosts are its neighbours' nodes
            assert np.array_equal(p.nodes, g.nodes[tuple(sl)])
            assert p.bc[direction] == (I.BC_BLOCK, I.BC_BLOCK)   # periodic parent: linked all round
            a0 += n
        nb = len(sizes)
        assert sorted(links) == sorted([(b, direction, 0, (b - 1) % nb) for b in range(nb)] +
                                       [(b, direction, 1, (b + 1) % nb) for b in range(nb)])
        q = np.random.default_rng(0).standard_normal((5,) + g.nodes.shape[1:])[:, 6:-6, 6:-6, 6:-6]
        q = np.ascontiguousarray(q)
        assert np.array_equal(np.concatenate(I.split_state(q, direction, sizes), axis=ax), q)


def test_split_grid_keeps_non_periodic_outer_sides():
    g = I.cylinder_ogrid((16, 12, 8), Lz=2.0, Gn=6)
    parts, links = I.split_grid(g, 1, (5, 7))        # radial split: wall side and far field stay
    assert parts[0].bc[1] == (g.bc[1][0], I.BC_BLOCK)
    assert parts[1].bc[1] == (I.BC_BLOCK, g.bc[1][1])
    assert sorted(links) == [(0, 1, 1, 1), (1, 1, 0, 0)]


def test_cgrid_wake_ghost_nodes_are_the_cut_partners():
    """Across the C-grid cut, ghost node (i, -1-m) is node (ni-1-i, m) for the wake cells."""
    ni, nj, nk, Gn = 48, 24, 16, 12
    g = I.cgrid_wing(n=(ni, nj, nk), Gn=Gn)
    assert g.cut > 0 and g.bc[1][0] == I.BC_CUT
    for i in list(range(-Gn, g.cut)) + list(range(ni - g.cut, ni + Gn)):
        for m in range(Gn):
            assert np.array_equal(g.nodes[:, :, Gn - 1 - m, i + Gn], g.nodes[:, :, Gn + m, ni - 1 - i + Gn])
