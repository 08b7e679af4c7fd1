"""Periodic neighbour pairs (the paper's linked-list cell decomposition and
adjacency list, Sec. 2.4, done here by brute force and by an independent
cell list).

Reading of the pair set (the paper only says pairs lie "within a finite cutoff
distance", Sec. 2.1):
  * positions are wrapped per axis into [0, L): q = floor(r / L), w = r - q L,
    then w += L if w < 0, then w = 0 if w >= L (FP64, each operation rounded);
  * a pair is (i, j, n) with image vector n in Z^3, (j, n) != (i, 0);
    Delta_a = (w_j,a - w_i,a) + n_a L_a and
    d^2 = (Dx Dx + Dy Dy) + Dz Dz, every operation rounded to FP64, no fused
    multiply-add;
  * included iff d^2 < r_cut * r_cut (strict); several images of the same j,
    and images of i itself, are allowed when r_cut > L/2;
  * canonical order: ascending (i, j, n_x, n_y, n_z); the reverse of (i, j, n)
    is (j, i, -n).
"""
import math
import numpy as np


def wrap_positions(pos, lengths):
    L = np.asarray(lengths, dtype=np.float64)[None, :]
    q = np.floor(pos / L)
    w = pos - q * L
    w = np.where(w < 0.0, w + L, w)
    w = np.where(w >= L, 0.0, w)
    return w


def _image_range(lengths, r_cut):
    return [int(math.ceil(r_cut / float(L))) for L in lengths]


def _sort_pairs(i, j, n):
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], j, i))
    return i[order], j[order], n[order]


def pairs_bruteforce(pos, lengths, r_cut, rows=None):
    """All (i, j, n) by testing every j and every image n with |n_a| <= ceil(rc/L_a).

    rows: optional iterable of centre atoms i to enumerate (default all).
    Returns (i int64 (P,), j int64 (P,), n int64 (P,3)) in canonical order.
    """
    w = wrap_positions(np.asarray(pos, dtype=np.float64), lengths)
    L = np.asarray(lengths, dtype=np.float64)
    N = w.shape[0]
    nr = _image_range(L, r_cut)
    imgs = np.array([(a, b, c)
                     for a in range(-nr[0], nr[0] + 1)
                     for b in range(-nr[1], nr[1] + 1)
                     for c in range(-nr[2], nr[2] + 1)], dtype=np.int64)
    shift = imgs * L[None, :]                       # exact: |n| <= 2
    rc2 = r_cut * r_cut
    rows = np.arange(N) if rows is None else np.asarray(list(rows), dtype=np.int64)
    I, J, NN = [], [], []
    chunk = max(1, 2_000_000 // (N * len(imgs)))
    for s in range(0, len(rows), chunk):
        ii = rows[s:s + chunk]
        # (ci, N, nimg)
        dx = (w[None, :, 0] - w[ii, None, 0])[:, :, None] + shift[None, None, :, 0]
        dy = (w[None, :, 1] - w[ii, None, 1])[:, :, None] + shift[None, None, :, 1]
        dz = (w[None, :, 2] - w[ii, None, 2])[:, :, None] + shift[None, None, :, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        mask = d2 < rc2
        a, b, c = np.nonzero(mask)
        ci = ii[a]
        keep = ~((ci == b) & np.all(imgs[c] == 0, axis=1))
        I.append(ci[keep])
        J.append(b[keep])
        NN.append(imgs[c[keep]])
    i = np.concatenate(I) if I else np.zeros(0, np.int64)
    j = np.concatenate(J) if J else np.zeros(0, np.int64)
    n = np.concatenate(NN) if NN else np.zeros((0, 3), np.int64)
    return _sort_pairs(i.astype(np.int64), j.astype(np.int64), n.astype(np.int64))


def pairs_cells(pos, lengths, r_cut):
    """Same pair set via a linked-cell decomposition (O(N)); needs L >= 3 r_cut
    on every axis, otherwise falls back to brute force."""
    L = np.asarray(lengths, dtype=np.float64)
    ncell = np.floor(L / (r_cut * (1.0 + 1e-9))).astype(np.int64)
    if np.any(ncell < 3):
        return pairs_bruteforce(pos, lengths, r_cut)
    w = wrap_positions(np.asarray(pos, dtype=np.float64), L)
    N = w.shape[0]
    cidx = np.minimum((w / (L / ncell)[None, :]).astype(np.int64), ncell[None, :] - 1)
    flat = (cidx[:, 0] * ncell[1] + cidx[:, 1]) * ncell[2] + cidx[:, 2]
    nc_tot = int(ncell.prod())
    order = np.argsort(flat, kind="stable")
    counts = np.bincount(flat, minlength=nc_tot)
    start = np.concatenate([[0], np.cumsum(counts)])
    maxc = int(counts.max())
    # padded member table [cell, slot] -> atom (or -1)
    table = -np.ones((nc_tot, maxc), dtype=np.int64)
    slot = np.arange(N) - start[flat[order]]
    table[flat[order], slot] = order
    cx, cy, cz = np.unravel_index(np.arange(nc_tot), tuple(ncell))
    rc2 = r_cut * r_cut
    I, J, NN = [], [], []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for oz in (-1, 0, 1):
                tx, ty, tz = cx + ox, cy + oy, cz + oz
                nx, ny, nz = tx // ncell[0], ty // ncell[1], tz // ncell[2]
                other = ((tx % ncell[0]) * ncell[1] + ty % ncell[1]) * ncell[2] + tz % ncell[2]
                A = table                        # (nc, maxc) centres
                B = table[other]                 # (nc, maxc) candidates
                valid = (A[:, :, None] >= 0) & (B[:, None, :] >= 0)
                Ai = np.where(A < 0, 0, A)
                Bj = np.where(B < 0, 0, B)
                sh = np.stack([nx, ny, nz], axis=1) * L[None, :]   # (nc, 3)
                dx = (w[Bj, 0][:, None, :] - w[Ai, 0][:, :, None]) + sh[:, 0, None, None]
                dy = (w[Bj, 1][:, None, :] - w[Ai, 1][:, :, None]) + sh[:, 1, None, None]
                dz = (w[Bj, 2][:, None, :] - w[Ai, 2][:, :, None]) + sh[:, 2, None, None]
                d2 = (dx * dx + dy * dy) + dz * dz
                img0 = (nx == 0) & (ny == 0) & (nz == 0)
                same = (Ai[:, :, None] == Bj[:, None, :]) & img0[:, None, None]
                m = valid & (d2 < rc2) & ~same
                c, a, b = np.nonzero(m)
                I.append(Ai[c, a])
                J.append(Bj[c, b])
                NN.append(np.stack([nx[c], ny[c], nz[c]], axis=1))
    i = np.concatenate(I)
    j = np.concatenate(J)
    n = np.concatenate(NN)
    return _sort_pairs(i.astype(np.int64), j.astype(np.int64), n.astype(np.int64))


def pairs_auto(pos, lengths, r_cut):
    """Brute force for small systems, the cell list otherwise (same pair set)."""
    n = len(pos)
    nimg = 1
    for r in _image_range(lengths, r_cut):
        nimg *= 2 * r + 1
    ncell = 1
    for L in lengths:
        ncell *= max(1, int(math.floor(float(L) / r_cut)))
    if n * n * nimg <= 4_000_000 or ncell > 4 * n:     # small or sparse: brute force
        return pairs_bruteforce(pos, lengths, r_cut)
    return pairs_cells(pos, lengths, r_cut)


def reverse_index(i, j, n, n_atoms):
    """rev[p] = index of (j, i, -n) for every pair p (pairs in canonical order)."""
    code = ((n[:, 0] + 2) * 25 + (n[:, 1] + 2) * 5 + (n[:, 2] + 2)).astype(np.int64)
    rcode = ((-n[:, 0] + 2) * 25 + (-n[:, 1] + 2) * 5 + (-n[:, 2] + 2)).astype(np.int64)
    key = (i * n_atoms + j) * 125 + code
    rkey = (j * n_atoms + i) * 125 + rcode
    rev = np.searchsorted(key, rkey)
    assert np.all(key[rev] == rkey), "pair set is not closed under reversal"
    return rev
