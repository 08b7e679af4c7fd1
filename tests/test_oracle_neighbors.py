"""Pins for the oracle's periodic pair list (Sec. 2.4 linked-list cells and
adjacency list; strict d^2 < r_cut^2 reading with all periodic images)."""
import numpy as np
import pytest

import synth
from oracle.neighbors import pairs_bruteforce, pairs_cells, reverse_index, wrap_positions


def _sc_lattice(n, a):
    g = np.arange(n) * a + 0.25 * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1), np.full(3, n * a)


@pytest.mark.parametrize("rc,per_atom", [(2.5, 6), (3.0, 18), (3.5, 26), (4.1, 32)])
def test_simple_cubic_shell_counts(rc, per_atom):
    # shells of a simple-cubic lattice (a = 2): 6 at 2, 12 at 2.83, 8 at 3.46, 6 at 4
    pos, L = _sc_lattice(6, 2.0)
    for fn in (pairs_bruteforce, pairs_cells):
        i, j, n = fn(pos, L, rc)
        assert np.all(np.bincount(i, minlength=len(pos)) == per_atom)


def test_single_atom_self_images():
    pos = np.array([[0.3, 1.1, 2.9]])
    L = np.array([3.0, 3.0, 3.0])
    i, j, n = pairs_bruteforce(pos, L, 3.5)           # six images at distance 3
    assert len(i) == 6 and np.all(j == 0)
    assert sorted(map(tuple, n)) == sorted([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])
    i, j, n = pairs_bruteforce(pos, L, 4.3)           # + 12 at 3*sqrt2 = 4.243
    assert len(i) == 18


def test_strict_cutoff():
    pos = np.array([[1.0, 1.0, 1.0], [3.0, 1.0, 1.0]])
    L = np.array([50.0, 50.0, 50.0])
    assert len(pairs_bruteforce(pos, L, 2.0)[0]) == 0
    assert len(pairs_bruteforce(pos, L, 2.0 + 1e-12)[0]) == 2


def test_wrapping_rules():
    L = np.array([4.0, 4.0, 4.0])
    w = wrap_positions(np.array([[-1e-17, 4.0, 9.5]]), L)
    assert np.all(w >= 0) and np.all(w < L)
    assert w[0, 1] == 0.0 and w[0, 2] == 1.5
    pos, sp, cell = synth.make_ammonia(16, 3)
    Ld = np.diag(cell)
    a = pairs_bruteforce(pos, Ld, 4.0)
    b = pairs_bruteforce(pos + 3 * Ld[None, :], Ld, 4.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_cells_equal_bruteforce_liquid():
    pos, sp, cell = synth.make_ammonia(108, 5)        # L = 17.4 A, 3 cells at rc 5
    L = np.diag(cell)
    a = pairs_bruteforce(pos, L, 5.0)
    b = pairs_cells(pos, L, 5.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_cells_equal_bruteforce_rows_6912():
    pos, sp, cell = synth.make_ammonia(1728, 0)
    L = np.diag(cell)
    i, j, n = pairs_cells(pos, L, 5.0)
    rows = [0, 1, 17, 4000, 6911]
    bi, bj, bn = pairs_bruteforce(pos, L, 5.0, rows=rows)
    sel = np.isin(i, rows)
    assert np.array_equal(i[sel], bi) and np.array_equal(j[sel], bj) and np.array_equal(n[sel], bn)


def test_reverse_is_involution_and_small_box_has_multi_images():
    pos, sp, cell = synth.make_ammonia(16, 0)         # 64 atoms, L = 8.73 < 2 * 5
    L = np.diag(cell)
    i, j, n = pairs_bruteforce(pos, L, 5.0)
    rev = reverse_index(i, j, n, len(pos))
    assert np.all(rev[rev] == np.arange(len(i)))
    assert np.all(i[rev] == j) and np.all(j[rev] == i) and np.all(n[rev] == -n)
    assert not np.any(i == j)                         # L = 8.73 > rc: no self-image
    # several images of the same partner appear as separate pairs
    key = i * len(pos) + j
    assert len(np.unique(key)) < len(key)
