"""GPU NVE velocity Verlet (Eq. 1, Sec. 3.2), Nose-Hoover NVT and the >5 sigma
outlier count (Fig. 1 caption) vs the oracle."""
import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from oracle.md import kinetic_energy, nose_hoover, outlier_count, velocity_verlet
from oracle.model import OracleModel
from tests.conftest import energy_scale

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])


def test_outlier_count_matches_bruteforce():
    cfg = synth.TINY
    ctx = al.allegro_create(synth.make_blob(cfg, 42), MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    rng = np.random.default_rng(0)
    for n in (1, 7, 1000, 100_000):
        F = rng.standard_t(3, size=(n, 3)).astype(np.float32)
        for thr in (5.0, 2.0):
            c = al.allegro_outlier_count(ctx, torch.tensor(F, device="cuda"), thr)
            f = F.astype(np.float64).ravel()
            sigma = np.sqrt(np.mean(f * f))
            near = np.abs(np.abs(f) - thr * sigma) <= 1e-9 * thr * sigma
            ref = outlier_count(F, thr)
            assert abs(c - ref) <= int(near.sum())
    al.allegro_destroy(ctx)


def test_tiny_nve_matches_oracle_trajectory():
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    orc = OracleModel(blob)
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    v0 = synth.make_velocities(sp, 200.0, 1)
    n = 20
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    en = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    al.allegro_md_step_nve(ctx, 0.5, n, out, en)
    P = np.zeros((len(pos), 3))
    V = np.zeros((len(pos), 3))
    step = al.allegro_md_get_state(ctx, P, V)
    assert step == n
    ref = velocity_verlet(lambda p: orc.energy_forces(p, sp, L)[:2], pos, v0, MASS[sp], L, 0.5, n)
    en = en.cpu().numpy()
    # FP32 forces drive an FP64 integrator: trajectories agree to ~1e-6 over 20 steps
    d = P - ref["pos"]
    d -= np.round(d / L) * L
    assert np.abs(d).max() < 1e-5
    assert np.abs(V - ref["vel"]).max() < 1e-5
    np.testing.assert_allclose(en[:, 0], ref["epot"], rtol=0, atol=1e-4 * abs(ref["epot"]).max())
    np.testing.assert_allclose(en[:, 1], ref["ekin"], rtol=1e-5, atol=1e-7)
    assert np.array_equal(out.cpu().numpy(), ref["outliers"]) or \
        np.abs(out.cpu().numpy() - ref["outliers"]).max() <= 1
    assert abs(kinetic_energy(V, MASS[sp]) - en[-1, 1]) < 1e-9 * en[-1, 1]
    al.allegro_destroy(ctx)


def test_md_6912_energy_conservation_and_resume():
    cfg = synth.MAIN
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(1728, 0)
    v0 = synth.make_velocities(sp, 200.0, 1)
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    e1 = np.zeros((50, 3))
    o1 = np.zeros(50, np.int64)
    al.allegro_md_step_nve(ctx, 0.25, 50, o1, e1)
    kT = 8.617333e-5 * 200.0
    assert np.abs(e1[:, 2] - e1[0, 2]).max() / (len(sp) * kT) < 0.05
    assert np.all(o1 >= 0) and np.all(o1 < 3 * len(sp))
    # resume: two calls of 25 steps equal one call of 50 (bitwise, deterministic kernels)
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    e2 = np.zeros((25, 3))
    al.allegro_md_step_nve(ctx, 0.25, 25, None, e2)
    e3 = np.zeros((25, 3))
    al.allegro_md_step_nve(ctx, 0.25, 25, None, e3)
    assert np.array_equal(np.concatenate([e2, e3]), e1)
    al.allegro_destroy(ctx)


def test_tiny_nvt_matches_oracle_trajectory():
    """A hot start (400 K) thermostatted to 200 K with a 10 fs period: the
    thermostat acts within the 20 steps, and positions, velocities, energies,
    the extended energy H and the thermostat variable follow the oracle."""
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    orc = OracleModel(blob)
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    v0 = synth.make_velocities(sp, 400.0, 1)
    n, T, tau = 20, 200.0, 10.0
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    assert al.allegro_md_get_thermostat(ctx) == (0.0, 0.0)
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    en = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    al.allegro_md_step_nvt(ctx, 0.5, n, T, tau, out, en)
    P = np.zeros((len(pos), 3))
    V = np.zeros((len(pos), 3))
    assert al.allegro_md_get_state(ctx, P, V) == n
    xi, eta = al.allegro_md_get_thermostat(ctx)
    ref = nose_hoover(lambda p: orc.energy_forces(p, sp, L)[:2], pos, v0, MASS[sp], L, 0.5, n, T, tau)
    en = en.cpu().numpy()
    d = P - ref["pos"]
    d -= np.round(d / L) * L
    assert np.abs(d).max() < 1e-5
    assert np.abs(V - ref["vel"]).max() < 1e-5
    assert abs(ref["xi"]) > 1e-3 and abs(xi - ref["xi"]) <= 1e-4 * abs(ref["xi"])
    assert abs(eta - ref["eta"]) <= 1e-4 * abs(ref["eta"])
    np.testing.assert_allclose(en[:, 1], ref["ekin"], rtol=1e-5, atol=1e-7)
    scale = abs(ref["epot"]).max()
    np.testing.assert_allclose(en[:, 0], ref["epot"], rtol=0, atol=1e-4 * scale)
    np.testing.assert_allclose(en[:, 3], ref["hext"], rtol=0, atol=1e-4 * scale)
    assert abs(kinetic_energy(V, MASS[sp]) - en[-1, 1]) < 1e-9 * en[-1, 1]
    al.allegro_destroy(ctx)


def test_nvt_conserves_extended_energy_and_cools():
    """200 steps from 400 K to 200 K: the total energy falls by far more than
    the extended energy H moves, and the thermostat state carries over from
    one call to the next (two calls of 100 steps equal one of 200)."""
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    v0 = synth.make_velocities(sp, 400.0, 1)
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    e1 = np.zeros((200, 4))
    al.allegro_md_step_nvt(ctx, 0.25, 200, 200.0, 10.0, None, e1)
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    a, b = np.zeros((100, 4)), np.zeros((100, 4))
    al.allegro_md_step_nvt(ctx, 0.25, 100, 200.0, 10.0, None, a)
    al.allegro_md_step_nvt(ctx, 0.25, 100, 200.0, 10.0, None, b)
    assert np.array_equal(np.vstack([a, b]), e1)
    dH = np.abs(e1[:, 3] - e1[0, 3]).max()
    dE = e1[0, 2] - e1[:, 2].min()
    assert dE > 0 and dH < 0.1 * dE
    al.allegro_destroy(ctx)


# force difference between the two runs: FP32, the summation order of the
# per-atom sums (up to 100 terms, 2^-24 each: 1e-6 of max |F| ~ 5 eV/A);
# split mode, each run within the method's 2e-3 eV/A of the exact forces
@pytest.mark.parametrize("prec,dF", [(al.ALLEGRO_FP32, 5e-6), (al.ALLEGRO_FP16_SPLIT, 4e-3)], ids=["fp32", "fp16split"])
def test_verlet_skin_matches_rebuild_every_step(prec, dF):
    """Verlet-skin reuse (allegro_set_skin): the list built with r_cut + skin
    is kept until an atom has moved by more than skin/2.  Pairs beyond r_cut
    contribute exactly zero, so the trajectory equals the one with a rebuild at
    every step up to the summation order of the per-atom sums (the extra pairs
    shift tile boundaries).  A force difference dF moves the lightest atom
    (1.008 amu) by at most kappa dF t^2 / (2 m) over t = 40 x 0.25 fs, times
    4 for the divergence of neighbouring trajectories (as in the NVE
    trajectory test), and changes its velocity by kappa dF t / m times 4.
    A wide skin rebuilds rarely, a narrow one often; a missed pair or a stale
    image code would move atoms by far more."""
    kappa, t, m = 9.648533e-3, 10.0, 1.008
    tol, tolv = 4 * kappa * dF * t * t / (2 * m), 4 * kappa * dF * t / m
    cfg = synth.MAIN
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    pos, sp, cell = synth.make_ammonia(108, 0)
    v0 = synth.make_velocities(sp, 200.0, 1)
    n = 40
    out = {}
    for skin in (0.0, 0.6, 0.02):
        ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
        try:
            al.allegro_set_md_precision(ctx, prec)
            al.allegro_set_skin(ctx, skin)
            al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
            np0 = al.allegro_query(ctx, al.ALLEGRO_Q_N_PAIRS)
            e = np.zeros((n, 3))
            al.allegro_md_step_nve(ctx, 0.25, n, None, e)
            P, V = np.zeros_like(pos), np.zeros_like(pos)
            al.allegro_md_get_state(ctx, P, V)
            out[skin] = (P, V, e, np0, al.allegro_query(ctx, al.ALLEGRO_Q_REBUILDS))
        finally:
            al.allegro_destroy(ctx)
    L = np.diag(cell)
    for skin in (0.6, 0.02):
        d = out[skin][0] - out[0.0][0]
        d -= np.round(d / L) * L
        assert np.abs(d).max() <= tol, (skin, np.abs(d).max())
        assert np.abs(out[skin][1] - out[0.0][1]).max() <= tolv
    assert out[0.6][3] > out[0.0][3]                 # the skin list holds more pairs
    # the synthetic system heats fast (fastest atoms ~0.03 A/fs): the wide skin
    # still saves most builds, the narrow one rebuilds far more often
    assert 1 <= out[0.6][4] < n // 2
    assert out[0.6][4] < out[0.02][4] <= n
    with pytest.raises(al.AllegroError):
        ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
        try:
            al.allegro_set_skin(ctx, -1.0)
        finally:
            al.allegro_destroy(ctx)
