"""torch.autograd glue (paper_2303_08169_gb300.torch_ops) over the library's
hand-written adjoints: gradients equal the library's forces and weight
gradient, match the oracle, follow the chain rule, and drive a torch
optimizer."""
import json

import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from paper_2303_08169_gb300 import torch_ops
from oracle.model import OracleModel
from oracle.train import flat_params, loss_and_grad
from tests.conftest import GOLDEN, energy_scale
from tests.test_gpu_train import _structs

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])


def test_energy_gradient_is_minus_the_library_forces():
    cfg = synth.MAIN
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(108, 5)
    sp_d = torch.tensor(sp, dtype=torch.int32, device="cuda")
    r = torch.tensor(pos, device="cuda", requires_grad=True)
    E = torch_ops.energy(ctx, r, sp_d, cell)
    (g,) = torch.autograd.grad(E, r)
    F = torch.empty((len(pos), 3), dtype=torch.float32, device="cuda")
    E1 = al.allegro_energy_forces(ctx, torch.tensor(pos, device="cuda"), sp_d, cell, F)
    assert E.item() == E1
    assert torch.equal(g, -F.double())
    Er, Fr, _, _ = OracleModel(blob).energy_forces(pos, sp, np.diag(cell))
    assert abs(E.item() - Er) <= 1e-5 * abs(Er)
    assert np.abs(g.cpu().numpy() + Fr).max() <= 1e-5 * np.abs(Fr).max()
    # chain rule through ordinary torch ops
    r2 = torch.tensor(pos, device="cuda", requires_grad=True)
    y = 3.0 * torch_ops.energy(ctx, r2, sp_d, cell) + (r2 * r2).sum()
    y.backward()
    assert torch.allclose(r2.grad, -3.0 * F.double() + 2.0 * r2.detach(), rtol=0, atol=1e-12)
    al.allegro_destroy(ctx)


def test_batch_loss_gradient_and_torch_optimizer():
    cfg = synth.TINY
    scales = json.load(open(f"{GOLDEN}/energy_scale.json"))
    blob = synth.make_blob(cfg, 42, sigma=scales["tiny"]["sigma"])
    tea = OracleModel(synth.make_blob(cfg, 43, sigma=scales["tiny_teacher"]["sigma"]))
    stu = OracleModel(blob)
    structs = _structs(tea)
    ctx = al.allegro_create(blob, synth.MASS_AMU, cfg.r_cut, cfg.l_max, cfg.n_layers)
    b, keep = al.make_batch(structs)
    n = al.allegro_query(ctx, al.ALLEGRO_Q_N_PARAMS)
    w0 = np.zeros(n, np.float32)
    al.allegro_get_weights(ctx, w0)
    w = torch.tensor(w0, device="cuda", requires_grad=True)
    L = torch_ops.batch_loss(ctx, w, b)
    L.backward()
    g = torch.empty(n, dtype=torch.float32, device="cuda")
    L1 = al.allegro_loss_grad(ctx, b, 1.0, 100.0, g)
    assert L.item() == L1
    # the weight-gradient reductions add chunk partials with atomics: equal
    # up to FP32 summation order
    assert torch.linalg.norm(w.grad - g) <= 1e-5 * torch.linalg.norm(g)
    lref, gref = loss_and_grad(stu, flat_params(stu).numpy(), structs, 1.0, 100.0)
    gref = np.asarray(gref)
    assert abs(L.item() - lref) <= 1e-5 * lref
    assert np.linalg.norm(w.grad.cpu().numpy() - gref) <= 2e-3 * np.linalg.norm(gref)
    # a torch optimizer on the library's loss and gradient
    opt = torch.optim.Adam([w], lr=2e-3)
    losses = []
    for _ in range(20):
        opt.zero_grad()
        loss = torch_ops.batch_loss(ctx, w, b)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < losses[0]
    al.allegro_destroy(ctx)
