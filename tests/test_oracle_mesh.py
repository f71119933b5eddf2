"""Pins for oracle.mesh: numbering round trips and refinement (Sec. 2.1)."""
import numpy as np

from oracle.mesh import TensorMesh, local_multi_indices


def test_cell_numbering_round_trip_and_x_fastest():
    m = TensorMesh([np.ones(3), np.ones(4), np.ones(2)])
    assert m.num_cells == 24
    for c in range(m.num_cells):
        assert m.cell_index(m.cell_multi(c)) == c
    assert m.cell_multi(1) == (1, 0, 0)
    assert m.cell_multi(3) == (0, 1, 0)


def test_local_multi_index_order_matches_eq_multiindex():
    # i = sum_t i_t (k+1)^(t-1): first index fastest
    k, d = 2, 3
    for i, im in enumerate(local_multi_indices(k, d)):
        assert i == im[0] + 3 * im[1] + 9 * im[2]


def test_refine_halves_widths_and_keeps_domain():
    rng = np.random.default_rng(0)
    w = [rng.uniform(0.5, 1.5, 3), rng.uniform(0.5, 1.5, 2)]
    m = TensorMesh(w)
    f = m.refine()
    assert f.ncells == (6, 4)
    for t in range(2):
        assert np.allclose(f.widths[t][0::2], 0.5 * w[t])
        assert np.isclose(f.widths[t].sum(), w[t].sum())
