"""Tensor-core pair passes (tcgen05, BF16 or FP16 operands, FP32 accumulation)
for the 2-layer l_max 2 model.

Two references:
  * the oracle in operand-emulation mode (every per-pair GEMM input and
    pre-scaled weight rounded to the same 16-bit type, FP64 accumulation):
    the tensor-core energies must match it to FP32-accumulation level, which
    pins the kernels themselves;
  * the exact FP64 oracle: the force error that the operand precision
    implies for this seeded model, stated and bounded.
Measured on GB300 (6,912 atoms): BF16 max |dF| 4.0e-2, rms 1.1e-2 eV/A;
FP16 max 3.0e-3, rms 7.3e-4 eV/A; FP16_SPLIT max 7.6e-4 eV/A (RMS force
1 eV/A).  Energy vs the emulating oracle: the path stores x^k, V^k and the
layer scalars in FP16 between passes, which the emulation rounds the same way;
values that the GPU knows only to FP32 accumulation (or, in the split mode, to
the ~1e-6 of FP16 hi/lo pairs whose lo part is subnormal) round to the other
FP16 neighbour when they lie that close to a midpoint, and the emulation
cannot follow those flips: measured 5.7e-6 (BF16), 4.7e-6 (FP16) and 5.3e-5
(FP16_SPLIT) relative at 432 atoms.  Bounds below carry margin, except the
split mode's max |dF|, which is the 2e-3 eV/A acceptance bound of the
mixed-precision path."""
import dataclasses

import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from oracle.model import OracleModel
from tests.conftest import energy_scale

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])
MODES = {"bf16": (al.ALLEGRO_BF16, dict(erel=5e-5, ei=1e-2, fmax=6e-2, frms=1.5e-2)),
         "fp16": (al.ALLEGRO_FP16, dict(erel=2e-5, ei=2e-3, fmax=5e-3, frms=1.2e-3)),
         "fp16split": (al.ALLEGRO_FP16_SPLIT, dict(erel=1.5e-4, ei=2e-3, fmax=2e-3, frms=5e-4))}


@pytest.fixture(scope="module")
def main():
    cfg = synth.MAIN
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    yield ctx, blob
    al.allegro_destroy(ctx)


def _gpu(ctx, pos, sp, cell, prec):
    N = len(pos)
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    Ei = torch.empty(N, dtype=torch.float64, device="cuda")
    E = al.allegro_energy_forces(ctx, torch.tensor(pos, device="cuda"), torch.tensor(sp, device="cuda"), cell,
                                 F, Ei, prec)
    return E, F.cpu().numpy().astype(np.float64), Ei.cpu().numpy()


@pytest.mark.parametrize("mode", ["bf16", "fp16", "fp16split"])
@pytest.mark.parametrize("n_mol", [108, 1728])
def test_tensorcore_vs_emulating_and_exact_oracle(main, mode, n_mol):
    ctx, blob = main
    prec, tol = MODES[mode]
    pos, sp, cell = synth.make_ammonia(n_mol, 0)
    L = np.diag(cell)
    E, F, Ei = _gpu(ctx, pos, sp, cell, prec)
    Er, Fr, Eir, pairs = OracleModel(blob).energy_forces(pos, sp, L)
    Ee, Fe, Eie, _ = OracleModel(blob, emulate=mode).energy_forces(pos, sp, L, pairs=pairs)
    assert abs(E - Ee) <= tol["erel"] * abs(Ee)
    assert np.abs(Ei - Eie).max() <= tol["ei"]
    d = F - Fr
    assert np.abs(d).max() <= tol["fmax"]
    assert np.sqrt(np.mean(d * d)) <= tol["frms"]
    E2, F2, _ = _gpu(ctx, pos, sp, cell, prec)
    assert E2 == E and np.array_equal(F2, F)          # bitwise rerun


@pytest.mark.parametrize("mode", ["bf16", "fp16", "fp16split"])
def test_tensorcore_sampled_atoms_110592(main, mode):
    ctx, blob = main
    prec, tol = MODES[mode]
    pos, sp, cell = synth.make_ammonia(27648, 0)
    E, F, Ei = _gpu(ctx, pos, sp, cell, prec)
    orc = OracleModel(blob)
    rng = np.random.default_rng(5)
    for k in rng.choice(len(pos), 8, replace=False):
        ek, fk = orc.local_energy_force(pos, sp, np.diag(cell), int(k))
        assert np.abs(F[k] - fk).max() <= tol["fmax"]
    assert np.abs(F.sum(0)).max() <= 1e-2 * np.sqrt(len(pos))


def test_tensorcore_md_and_unsupported_model(main):
    ctx, blob = main
    pos, sp, cell = synth.make_ammonia(1728, 0)
    v0 = synth.make_velocities(sp, 200.0, 1)
    al.allegro_set_md_precision(ctx, al.ALLEGRO_BF16)
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    e = np.zeros((40, 3))
    al.allegro_md_step_nve(ctx, 0.25, 40, None, e)
    kT = 8.617333e-5 * 200.0
    assert np.abs(e[:, 2] - e[0, 2]).max() / (len(sp) * kT) < 0.05
    al.allegro_set_md_precision(ctx, al.ALLEGRO_FP32)
    tiny = synth.TINY
    tctx = al.allegro_create(synth.make_blob(tiny, 42), MASS, tiny.r_cut, tiny.l_max, tiny.n_layers)
    p, s, c = synth.make_ammonia(16, 0)
    with pytest.raises(al.AllegroError) as err:
        al.allegro_energy_forces(tctx, p, s.astype(np.int32), c, None, None, al.ALLEGRO_BF16)
    assert err.value.code == 10
    al.allegro_destroy(tctx)


@pytest.mark.parametrize("mode", ["fp16", "fp16split"])
def test_tensorcore_three_layers(mode):
    """Three layers run the inner-layer passes twice (k = 1, 2): pass B1^T of
    k = 2 writes dV^1 instead of the embedding adjoint.  The deeper model makes
    the FP16 storage roundings more sensitive to their inputs: the emulating
    oracle itself moves by 1.4e-6 relative in energy and 8e-4 eV/A in force
    under 1e-8 A of random position noise (1e-7 and 2.7e-5 at 1e-10 A), and
    the kernels' FP32 pair separations differ from FP64 by ~1e-7 A, so the
    energy bound against the emulation is 1e-4 relative here."""
    cfg = dataclasses.replace(synth.MAIN, n_layers=3)
    blob = synth.make_blob(cfg, 44, sigma=energy_scale("main"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    try:
        prec, tol = MODES[mode]
        pos, sp, cell = synth.make_ammonia(108, 0)
        E, F, Ei = _gpu(ctx, pos, sp, cell, prec)
        Er, Fr, _, pairs = OracleModel(blob).energy_forces(pos, sp, np.diag(cell))
        Ee, Fe, _, _ = OracleModel(blob, emulate=mode).energy_forces(pos, sp, np.diag(cell), pairs=pairs)
        E32, F32, _ = _gpu(ctx, pos, sp, cell, al.ALLEGRO_FP32)
    finally:
        al.allegro_destroy(ctx)
    assert abs(E32 - Er) <= 1e-5 * abs(Er) and np.abs(F32 - Fr).max() <= 1e-4 * max(1.0, np.abs(Fr).max())
    assert abs(E - Ee) <= max(tol["erel"], 1e-4) * abs(Ee)
    d = F - Fe
    assert np.abs(d).max() <= tol["fmax"] and np.sqrt(np.mean(d * d)) <= tol["frms"]
    assert np.abs(F - Fr).max() <= 2 * tol["fmax"]     # one more layer of operand rounding


def test_tensorcore_wait_timeout_is_reported(main):
    """Failure detection without a GPU fault: with the weight copies of the
    tensor-core passes withheld (nothing in flight), their bounded mbarrier
    waits run out; the entry points must report ALLEGRO_E_TIMEOUT instead of
    returning stale energies, the MD step must restore its starting state, and
    the context must work normally once the injection is lifted."""
    ctx, blob = main
    pos, sp, cell = synth.make_ammonia(108, 0)
    E0, F0, _ = _gpu(ctx, pos, sp, cell, al.ALLEGRO_FP16_SPLIT)
    v0 = synth.make_velocities(sp, 200.0, 1)
    try:
        al.allegro_debug_inject_wait_timeout(True)
        with pytest.raises(al.AllegroError) as err:
            _gpu(ctx, pos, sp, cell, al.ALLEGRO_FP16_SPLIT)
        assert err.value.code == 8
        al.allegro_debug_inject_wait_timeout(False)
        al.allegro_set_md_precision(ctx, al.ALLEGRO_FP16_SPLIT)
        al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
        al.allegro_md_step_nve(ctx, 0.25, 2)
        r1, v1 = np.zeros_like(pos), np.zeros_like(pos)
        step1 = al.allegro_md_get_state(ctx, r1, v1)
        al.allegro_debug_inject_wait_timeout(True)
        with pytest.raises(al.AllegroError) as err:
            al.allegro_md_step_nve(ctx, 0.25, 3)
        assert err.value.code == 8
    finally:
        al.allegro_debug_inject_wait_timeout(False)
    r2, v2 = np.zeros_like(pos), np.zeros_like(pos)
    step2 = al.allegro_md_get_state(ctx, r2, v2)
    assert step2 == step1 and np.array_equal(r1, r2) and np.array_equal(v1, v2)
    al.allegro_md_step_nve(ctx, 0.25, 1)                  # the MD state still steps
    al.allegro_set_md_precision(ctx, al.ALLEGRO_FP32)
    E1, F1, _ = _gpu(ctx, pos, sp, cell, al.ALLEGRO_FP16_SPLIT)
    assert E1 == E0 and np.array_equal(F1, F0)
