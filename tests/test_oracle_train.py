"""Pins for the oracle's loss, weight gradient, Adam and SAM step (Eq. 3,
Table 5)."""
import math

import numpy as np
import pytest

import synth
from oracle.model import OracleModel
from oracle.train import adam_update, flat_params, loss_and_grad, loss_scan, sam_step, sharpness

MICRO = synth.ModelConfig(r_cut=4.0, l_max=1, n_layers=2, n_channels=2,
                          latent=(6, 6), energy=(4,), avg_num_neighbors=5.0,
                          sigma=(1.5, 0.8), mu=(0.1, -0.2))


def _batch(model, targets_from=None, n=2):
    out = []
    for b in range(n):
        pos, sp, cell = synth.make_ammonia(4 + 2 * b, 100 + b)
        L = np.diag(cell) * 0.85
        src = targets_from or model
        E, F, _, _ = src.energy_forces(pos, sp, L)
        out.append(dict(pos=pos, species=sp, lengths=L, e_target=E, f_target=F))
    return out


@pytest.fixture(scope="module")
def micro():
    return OracleModel(synth.make_blob(MICRO, 9))


def test_loss_normalisation_closed_form(micro):
    batch = _batch(micro)
    w = flat_params(micro).numpy()
    dE = [0.3, -1.1]
    dF = 0.05
    for s, e in zip(batch, dE):
        s["e_target"] = s["e_target"] - e
        s["f_target"] = s["f_target"] - dF
    loss, _ = loss_and_grad(micro, w, batch, 1.0, 100.0, need_grad=False)
    ntot = sum(len(s["species"]) for s in batch)
    ref = (sum((e / len(s["species"])) ** 2 for s, e in zip(batch, dE)) / 2
           + 100.0 * (3 * ntot * dF * dF) / (3 * ntot))
    assert abs(loss - ref) < 1e-12 * ref


def test_weight_gradient_finite_differences(micro):
    teacher = OracleModel(synth.make_blob(MICRO, 10))
    batch = _batch(micro, teacher)
    w = flat_params(micro).numpy()
    loss, g = loss_and_grad(micro, w, batch)
    rng = np.random.default_rng(0)
    h = 1e-4
    for k in rng.choice(len(w), 25, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (loss_and_grad(micro, wp, batch, need_grad=False)[0]
              - loss_and_grad(micro, wm, batch, need_grad=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(g[k]), 1e-3 * np.abs(g).max())


def test_adam_first_step_closed_form():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    z = np.zeros(3)
    w1, m, v, t = adam_update(w, g, z, z, 0, lr=2e-3)
    np.testing.assert_allclose(w1, w - 2e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert t == 1


def test_sam_special_cases(micro):
    teacher = OracleModel(synth.make_blob(MICRO, 10))
    batch = _batch(micro, teacher)
    w = flat_params(micro).numpy()
    z = np.zeros_like(w)
    # rho = 0: exactly the base Adam step at w
    w1, st, l0, l1, eps = sam_step(micro, w, batch, 0.0, 2e-3, (z, z, 0))
    _, g = loss_and_grad(micro, w, batch)
    w_ref, *_ = adam_update(w, g, z, z, 0, 2e-3)
    np.testing.assert_array_equal(w1, w_ref)
    assert l0 == l1
    # ||eps|| = rho
    w1, st, l0, l1, eps = sam_step(micro, w, batch, 0.05, 2e-3, (z, z, 0))
    assert abs(np.linalg.norm(eps) - 0.05) < 1e-14
    assert l1 > l0                           # an ascent step raises the loss
    # student == teacher: zero loss, zero gradient, zero ascent step
    batch_self = _batch(micro, micro)
    w2, st, l0, l1, eps = sam_step(micro, w, batch_self, 0.05, 2e-3, (z, z, 0))
    assert l0 < 1e-26 and np.all(eps == 0)


def test_loss_scan_base_point_closed_form(micro):
    """Scale 0 gives the loss at w itself, here a closed form (targets shifted
    by known amounts, as in the normalisation test)."""
    batch = _batch(micro)
    w = flat_params(micro).numpy()
    dE, dF = [0.3, -1.1], 0.05
    for s, e in zip(batch, dE):
        s["e_target"] = s["e_target"] - e
        s["f_target"] = s["f_target"] - dF
    ntot = sum(len(s["species"]) for s in batch)
    ref = (sum((e / len(s["species"])) ** 2 for s, e in zip(batch, dE)) / 2 + 100.0 * dF * dF)
    d = np.random.default_rng(1).normal(size=w.shape)
    out = loss_scan(micro, w, d, [0.0, 0.0], batch)
    assert np.all(np.abs(out - ref) < 1e-12 * ref)


def test_loss_scan_follows_the_gradient(micro):
    """Along a direction d the scan's central difference is the directional
    derivative g.d of the finite-difference-pinned gradient; shared and
    per-point directions agree."""
    teacher = OracleModel(synth.make_blob(MICRO, 10))
    batch = _batch(micro, teacher)
    w = flat_params(micro).numpy()
    _, g = loss_and_grad(micro, w, batch)
    rng = np.random.default_rng(2)
    d = rng.normal(size=w.shape)
    d /= np.linalg.norm(d)
    h = 1e-4
    shared = loss_scan(micro, w, d, [h, -h], batch)
    rows = loss_scan(micro, w, np.vstack([d, d]), [h, -h], batch)
    assert np.array_equal(shared, rows)
    assert abs((shared[0] - shared[1]) / (2 * h) - float(g @ d)) <= 1e-5 * np.linalg.norm(g)


def test_sharpness_first_order(micro):
    """For a small radius the sharpness over the pair {eps, -eps} is
    |g.eps| + O(rho^2): the larger side of the directional derivative."""
    teacher = OracleModel(synth.make_blob(MICRO, 10))
    batch = _batch(micro, teacher)
    w = flat_params(micro).numpy()
    _, g = loss_and_grad(micro, w, batch)
    d = np.random.default_rng(3).normal(size=w.shape)
    rho = 1e-4
    eps = rho * d / np.linalg.norm(d)
    s = sharpness(micro, w, np.vstack([eps, -eps]), batch)
    assert abs(s - abs(float(g @ eps))) <= 1e-3 * abs(float(g @ eps)) + 1e-9
