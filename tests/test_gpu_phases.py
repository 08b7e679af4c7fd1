"""Per-kernel device times (allegro_phase_times) and the split-mode NVE loop on
the 2-layer l_max 2 model, 6,912 atoms."""
import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from tests.conftest import energy_scale

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])
PASSES = ["pass_a", "pass_b", "pass_c", "pass_b_adjoint", "pass_a_adjoint"]


@pytest.fixture(scope="module")
def main_6912():
    cfg = synth.MAIN
    ctx = al.allegro_create(synth.make_blob(cfg, 42, sigma=energy_scale("main")), MASS, cfg.r_cut, cfg.l_max,
                            cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(1728, 0)
    yield ctx, pos, sp, cell, synth.make_velocities(sp, 200.0, 1)
    al.allegro_destroy(ctx)


def _call_ms(ctx, pos, sp, cell, prec, n=5):
    F = torch.empty((len(sp), 3), dtype=torch.float32, device="cuda")
    p, s = torch.tensor(pos, device="cuda"), torch.tensor(sp, device="cuda", dtype=torch.int32)
    al.allegro_energy_forces(ctx, p, s, cell, F, None, prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        al.allegro_energy_forces(ctx, p, s, cell, F, None, prec)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


@pytest.mark.parametrize("prec", [al.ALLEGRO_FP32, al.ALLEGRO_FP16_SPLIT])
def test_every_pass_is_timed_and_the_phases_add_up(main_6912, prec):
    ctx, pos, sp, cell, v = main_6912
    al.allegro_set_md_precision(ctx, prec)
    al.allegro_md_init(ctx, pos, v, sp.astype(np.int32), cell)
    ph = al.allegro_phase_times(ctx, 5)
    for k in PASSES + ["neighbors", "forces"]:
        assert ph[k] > 0.0, k
    if prec != al.ALLEGRO_FP32:                       # the two kernels of each tensor-core layer pass
        for k in ["pass_b1", "pass_b2"]:
            assert ph[k] > 0.0, k
        assert ph["pass_b"] == pytest.approx(ph["pass_b1"] + ph["pass_b2"])
    total = sum(ph[k] for k in PASSES + ["neighbors", "forces"])
    call = _call_ms(ctx, pos, sp, cell, prec)         # + host copies and launch gaps
    assert 0.7 * call <= total <= 1.05 * call


def test_split_mode_nve(main_6912):
    ctx, pos, sp, cell, v = main_6912
    al.allegro_set_md_precision(ctx, al.ALLEGRO_FP16_SPLIT)
    al.allegro_md_init(ctx, pos, v, sp.astype(np.int32), cell)
    e = np.zeros((40, 3))
    outl = np.zeros(40, dtype=np.int64)
    al.allegro_md_step_nve(ctx, 0.25, 40, outl, e)
    kT = 8.617333e-5 * 200.0
    assert np.all(np.isfinite(e))
    assert np.abs(e[:, 2] - e[0, 2]).max() / (len(sp) * kT) < 0.05
    assert np.abs(e[:, 0] + e[:, 1] - e[:, 2]).max() <= 1e-9 * np.abs(e[:, 2]).max()
    assert outl.min() >= 0
    al.allegro_set_md_precision(ctx, al.ALLEGRO_FP32)
