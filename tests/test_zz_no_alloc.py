"""The allocation-free outlier count (allegro_outlier_count_noalloc), for
callers that cannot allocate device memory (a foreign allocator owning the
device, latency-bound loops), against the context-based
allegro_outlier_count on the same forces.  Integer counts must agree exactly,
on two calls in a row (the shared scratch keeps the previous call's contents
and must not leak into the next result).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])


def test_noalloc_matches_context_count_twice():
    cfg = synth.TINY
    ctx = al.allegro_create(synth.make_blob(cfg, 42), MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    rng = np.random.default_rng(11)
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    L = al.lib()
    for n, thr in ((100_000, 5.0), (3_001, 2.0)):
        F = torch.tensor(rng.standard_t(3, size=(n, 3)).astype(np.float32), device="cuda")
        ref = al.allegro_outlier_count(ctx, F, thr)
        for _ in range(2):
            out.fill_(-1)
            rc = L.allegro_outlier_count_noalloc(n, F.data_ptr(), thr, out.data_ptr(), None)
            assert rc == 0
            torch.cuda.synchronize()
            assert int(out.item()) == ref
    al.allegro_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = al.lib()
    F = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert L.allegro_outlier_count_noalloc((1 << 22) + 1, F.data_ptr(), 5.0, out.data_ptr(), None) == 1
    assert b"4194304" in L.allegro_last_error(None)
    assert L.allegro_outlier_count_noalloc(0, F.data_ptr(), 5.0, out.data_ptr(), None) == 1
