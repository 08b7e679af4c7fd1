"""GPU neighbour list vs the oracle's pair set: bit-exact (same pairs, same
images, same canonical order, reverse index an involution onto (j, i, -n))."""
import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from oracle.neighbors import pairs_bruteforce, pairs_cells, reverse_index

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])


def _ctx(cfg):
    return al.allegro_create(synth.make_blob(cfg, 42), MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)


def _gpu_pairs(ctx, pos, cell, device_input=True):
    p = torch.tensor(pos, device="cuda") if device_input else np.ascontiguousarray(pos)
    P = al.allegro_build_neighbors(ctx, p, cell)
    N = len(pos)
    row = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(P, 1), dtype=torch.int32, device="cuda")
    img = torch.empty((max(P, 1), 3), dtype=torch.int8, device="cuda")
    rev = torch.empty(max(P, 1), dtype=torch.int32, device="cuda")
    al.allegro_get_neighbors(ctx, row, col, img, rev)
    row = row.cpu().numpy().astype(np.int64)
    i = np.repeat(np.arange(N), np.diff(row))
    return i, col.cpu().numpy()[:P].astype(np.int64), img.cpu().numpy()[:P].astype(np.int64), \
        rev.cpu().numpy()[:P].astype(np.int64)


def _check(ctx, pos, cell, rc, ref=None):
    L = np.diag(cell)
    i, j, n, rev = _gpu_pairs(ctx, pos, cell)
    ri, rj, rn = ref if ref is not None else pairs_bruteforce(pos, L, rc)
    assert len(i) == len(ri)
    assert np.array_equal(i, ri) and np.array_equal(j, rj) and np.array_equal(n, rn)
    assert np.array_equal(rev, reverse_index(ri, rj, rn, len(pos)))
    return len(i)


def test_tiny_small_box_mode():
    ctx = _ctx(synth.TINY)
    pos, sp, cell = synth.make_ammonia(16, 0)          # L = 8.73 < 3 rc: all images
    assert _check(ctx, pos, cell, 4.0) > 1000
    al.allegro_destroy(ctx)


def test_multi_image_rc_above_half_box():
    ctx = _ctx(synth.MAIN)
    pos, sp, cell = synth.make_ammonia(16, 1)          # rc 5 > L/2 = 4.37
    i, j, n = pairs_bruteforce(pos, np.diag(cell), 5.0)
    assert len(np.unique(i * 64 + j)) < len(i)
    _check(ctx, pos, cell, 5.0)
    al.allegro_destroy(ctx)


def test_self_images_and_lattice_shells():
    ctx = _ctx(synth.MAIN)
    # one atom in a 3 A box: its six face images at 3 A are inside r_c = 5 (and 12 at 4.24)
    pos = np.array([[0.3, 1.1, 2.9]])
    cell = np.diag([3.0, 3.0, 3.0])
    assert _check(ctx, pos, cell, 5.0) == 18
    # simple-cubic lattice a = 2: shells |n|^2 = 1..6 hold 6, 12, 8, 6, 24, 24 sites (d <= 4.9 < 5)
    g = np.arange(10) * 2.0 + 0.5
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    cell = np.diag([20.0, 20.0, 20.0])
    i, j, n, rev = _gpu_pairs(ctx, pos, cell)
    assert np.all(np.bincount(i, minlength=len(pos)) == 80)
    al.allegro_destroy(ctx)


def test_cell_mode_432_and_wrapping_from_host_input():
    ctx = _ctx(synth.MAIN)
    pos, sp, cell = synth.make_ammonia(108, 5)          # 3 cells per axis
    pos = pos + np.array([17.0, -40.0, 3.5])            # far outside the box
    ref = pairs_bruteforce(pos, np.diag(cell), 5.0)
    i, j, n, rev = _gpu_pairs(ctx, pos, cell, device_input=False)
    assert np.array_equal(i, ref[0]) and np.array_equal(j, ref[1]) and np.array_equal(n, ref[2])
    al.allegro_destroy(ctx)


def test_6912_full_list():
    ctx = _ctx(synth.MAIN)
    pos, sp, cell = synth.make_ammonia(1728, 0)
    ref = pairs_cells(pos, np.diag(cell), 5.0)
    assert _check(ctx, pos, cell, 5.0, ref) == 361032
    al.allegro_destroy(ctx)


def test_110592_sampled_rows():
    ctx = _ctx(synth.MAIN)
    pos, sp, cell = synth.make_ammonia(27648, 0)
    L = np.diag(cell)
    i, j, n, rev = _gpu_pairs(ctx, pos, cell)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(len(pos), 64, replace=False))
    bi, bj, bn = pairs_bruteforce(pos, L, 5.0, rows=rows)
    sel = np.isin(i, rows)
    assert np.array_equal(i[sel], bi) and np.array_equal(j[sel], bj) and np.array_equal(n[sel], bn)
    # reverse index: involution mapping (i, j, n) -> (j, i, -n)
    assert np.all(rev[rev] == np.arange(len(i)))
    assert np.all(i[rev] == j) and np.all(n[rev] == -n)
    al.allegro_destroy(ctx)
