"""Pins for the oracle's operand-emulation modes (the reference that the
tensor-core path is checked against, beside the exact model).

The emulation (oracle/model.py) rounds GEMM operands, adjoint-GEMM gradient
operands and the per-pair values kept between passes.  These tests fix it
against things other than itself:
  * the rounding primitive and one emulated GEMM (forward and adjoint) against
    values worked out by hand from the FP16 / BF16 formats (10 / 7 fraction
    bits, round to nearest, ties to even);
  * with every rounding made an identity (float64), each mode is the exact
    model: a dropped scale, a transposed operand or a wrong fold of 1/sqrt(nu)
    or of the mixing normalisation breaks this;
  * the split mode leaves exactly the two-body MLP and the energy hidden layer
    unrounded and rounds the other groups like the FP16 mode;
  * storage rounding changes values but passes gradients through;
  * adjoint rounding changes forces but never energies.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle.model import OracleModel, RoundedLinear, round_to

F64 = torch.float64
MINI = synth.ModelConfig(r_cut=4.5, l_max=2, n_layers=2, n_channels=4, latent=(8, 8), energy=(8,),
                         avg_num_neighbors=7.0, sigma=(1.3, 0.7), mu=(0.25, -0.5))
BIG = np.array([60.0, 60.0, 60.0])
MODES = ["bf16", "fp16", "fp16split"]


def _cluster(n_mol=6, seed=2):
    pos, sp, _ = synth.make_ammonia(n_mol, seed)
    return pos - pos.mean(0) + 30.0, sp


def test_rounding_by_hand():
    # FP16 near 1 has spacing 2^-10: 1 + 2^-11 is a tie and goes to the even
    # neighbour 1; 1 + 3 2^-11 is a tie between 1 + 2^-10 (odd) and 1 + 2^-9
    # (even).  BF16 near 1 has spacing 2^-7.
    x = torch.tensor([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 0.1, 1.0 / 3.0, 70000.0], dtype=F64)
    h = round_to(x, torch.float16)
    assert h[0].item() == 1.0
    assert h[1].item() == 1.001953125
    assert h[2].item() == 0.0999755859375          # 1638 * 2^-14
    assert h[3].item() == 0.333251953125           # 1365 * 2^-12
    assert math.isinf(h[4].item())                 # above the FP16 range
    b = round_to(torch.tensor([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 70000.0], dtype=F64), torch.bfloat16)
    assert b[0].item() == 1.0 and b[1].item() == 1.015625
    assert b[2].item() == 70144.0                  # 137 * 2^9
    rep = torch.tensor([0.5, -2.75, 1024.0], dtype=F64)   # representable in both: unchanged
    assert torch.equal(round_to(rep, torch.float16), rep) and torch.equal(round_to(rep, torch.bfloat16), rep)


def test_rounded_gemm_by_hand():
    """y = q(x) q(W / sqrt(2))^T for x = [1, 2], W = [3, 5]:
    3/sqrt2 = 2.12132 -> FP16 1086 * 2^-9 = 2.12109375, BF16 136 * 2^-6 = 2.125;
    5/sqrt2 = 3.53553 -> FP16 1810 * 2^-9 = 3.53515625, BF16 226 * 2^-6 = 3.53125.
    Adjoint with dy = 0.1 (FP16 1638 * 2^-14): dx = q(dy) q(Ws)."""
    x = torch.tensor([[1.0, 2.0]], dtype=F64, requires_grad=True)
    Ws = torch.tensor([[3.0, 5.0]], dtype=F64) / math.sqrt(2.0)
    q16 = lambda t: round_to(t, torch.float16)
    y = RoundedLinear.apply(x, Ws, q16, q16, q16)
    assert y.item() == 9.19140625                  # 2.12109375 + 2 * 3.53515625
    (g,) = torch.autograd.grad(y, x, torch.tensor([[0.1]], dtype=F64))
    assert g[0, 0].item() == 1778868 / 2 ** 23    # 1638 * 1086 / (2^14 2^9)
    assert g[0, 1].item() == 2964780 / 2 ** 23    # 1638 * 1810 / (2^14 2^9)
    qb = lambda t: round_to(t, torch.bfloat16)
    assert RoundedLinear.apply(x.detach(), Ws, qb, qb, qb).item() == 9.1875


def test_storage_rounding_is_straight_through():
    m = OracleModel(synth.make_blob(MINI, 3), emulate="bf16")    # storage is FP16 in every mode
    x = torch.tensor([0.1, 1.0 / 3.0, 0.5], dtype=F64, requires_grad=True)
    y = m._qs(x)
    assert y.tolist() == [0.0999755859375, 0.333251953125, 0.5]
    (g,) = torch.autograd.grad((y * torch.tensor([2.0, 3.0, -1.0], dtype=F64)).sum(), x)
    assert g.tolist() == [2.0, 3.0, -1.0]


@pytest.mark.parametrize("l_max", [0, 1, 2])
@pytest.mark.parametrize("mode", MODES)
def test_identity_rounding_is_the_exact_model(mode, l_max):
    """At every l_max the tensor-core passes run (the mixing GEMM over the
    (pair, m) rows of each order's K-slice, the embedding width C (l_max + 1))."""
    import dataclasses
    blob = synth.make_blob(dataclasses.replace(MINI, l_max=l_max), 5)
    pos, sp = _cluster()
    E0, F0, Ei0, pairs = OracleModel(blob).energy_forces(pos, sp, BIG)
    m = OracleModel(blob, emulate=mode)
    m.op_dtype = m.adj_dtype = m.store_dtype = F64
    E, F, Ei, _ = m.energy_forces(pos, sp, BIG, pairs=pairs)
    assert abs(E - E0) <= 1e-13 * abs(E0)
    assert np.abs(Ei - Ei0).max() <= 1e-13 * np.abs(Ei0).max()
    assert np.abs(F - F0).max() <= 1e-12 * np.abs(F0).max()
    # and the real rounding does change the result (the emulation is active)
    E1, F1, _, _ = OracleModel(blob, emulate=mode).energy_forces(pos, sp, BIG, pairs=pairs)
    assert abs(E1 - E0) > 1e-9 * abs(E0) and np.abs(F1 - F0).max() > 1e-8


def test_split_mode_groups():
    """fp16split: the two-body MLP and the energy hidden layer are the exact
    model's; every other GEMM group is rounded exactly as in the FP16 mode."""
    cfg = synth.MAIN
    blob = synth.make_blob(cfg, 42)
    mx, m16, ms = OracleModel(blob), OracleModel(blob, emulate="fp16"), OracleModel(blob, emulate="fp16split")
    rng = np.random.default_rng(0)
    w = mx.w
    h = torch.tensor(rng.normal(size=(64, 12)), dtype=F64)
    tb = [w["twobody.0"], w["twobody.1"]]
    assert torch.equal(ms._mlp(h, tb, group="twobody"), mx._mlp(h, tb, group="twobody"))
    assert (m16._mlp(h, tb, group="twobody") - mx._mlp(h, tb, group="twobody")).abs().max() > 1e-5
    x = torch.tensor(rng.normal(size=(64, 128)), dtype=F64)
    en = [w["energy.0"]]
    assert torch.equal(ms._mlp(x, en, group="energy"), mx._mlp(x, en, group="energy"))
    assert (m16._mlp(x, en, group="energy") - mx._mlp(x, en, group="energy")).abs().max() > 1e-5
    xs = torch.tensor(rng.normal(size=(64, 176)), dtype=F64)
    lat = [w["layer1.latent.0"], w["layer1.latent.1"]]
    assert torch.equal(ms._mlp(xs, lat, group="latent"), m16._mlp(xs, lat, group="latent"))
    assert torch.equal(ms._qlin(x, w["embed"], group="embed"), m16._qlin(x, w["embed"], group="embed"))
    e_s = ms._qlin(x, w["layer1.env"], 1.0 / math.sqrt(ms.nu), group="env")
    assert torch.equal(e_s, m16._qlin(x, w["layer1.env"], 1.0 / math.sqrt(ms.nu), group="env"))
    # env folds 1/sqrt(nu) into the weights (with 1/sqrt(fan_in)) before rounding
    Ws = w["layer1.env"] * ((1.0 / math.sqrt(ms.nu)) / math.sqrt(128.0))
    assert torch.equal(e_s, round_to(x, torch.float16) @ round_to(Ws, torch.float16).T)


def test_adjoint_rounding_changes_forces_not_energies():
    blob = synth.make_blob(MINI, 5)
    pos, sp = _cluster()
    E0, F0, _, pairs = OracleModel(blob).energy_forces(pos, sp, BIG)
    m = OracleModel(blob, emulate="fp16")
    m.op_dtype = m.store_dtype = F64            # forward exact, adjoint operands FP16
    E, F, _, _ = m.energy_forces(pos, sp, BIG, pairs=pairs)
    assert abs(E - E0) <= 1e-13 * abs(E0)
    rel = np.abs(F - F0).max() / np.abs(F0).max()
    assert 1e-6 < rel < 1e-2                    # a few FP16 ulps (2^-11 = 4.9e-4) through the adjoint


def test_perturbation_hooks_act_only_when_set():
    blob = synth.make_blob(MINI, 5)
    pos, sp = _cluster()
    m = OracleModel(blob, emulate="fp16")
    E0, F0, _, pairs = m.energy_forces(pos, sp, BIG)
    E1, F1, _, _ = m.energy_forces(pos, sp, BIG, pairs=pairs)
    assert E0 == E1 and np.array_equal(F0, F1)
    m.perturb_value = lambda v: v * (1 + 1e-3)
    m.perturb_grad = lambda g: g * (1 + 1e-3)
    m.perturb_silu = lambda z: 1e-3 * z.abs()
    E2, F2, _, _ = m.energy_forces(pos, sp, BIG, pairs=pairs)
    assert E2 != E0 and not np.array_equal(F2, F0)
    mx = OracleModel(blob)                      # the exact model ignores value and gradient hooks
    mx.perturb_value = mx.perturb_grad = lambda v: v * 2.0
    Ex, Fx, _, _ = mx.energy_forces(pos, sp, BIG, pairs=pairs)
    Ex0, Fx0, _, _ = OracleModel(blob).energy_forces(pos, sp, BIG, pairs=pairs)
    assert Ex == Ex0 and np.array_equal(Fx, Fx0)
