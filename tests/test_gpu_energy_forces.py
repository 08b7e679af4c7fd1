"""GPU energy/forces (FP32 path) vs the FP64 oracle.

Tolerances (FP32 path): |dE| / |E| <= 1e-5 (or |dE| / (N rms E_i) when |E| is
small), max |dF| / max |F_ref| <= 1e-5, per-atom energies within
1e-5 * rms(E_i).  Covers the 1-layer l_max 1 model (passes A, C, A^T) and the
2-layer l_max 2 model (A, B, C, B^T, A^T), small boxes with several images of
one partner, tile-straddling rows, sampled atoms of the 110,592-atom
system, the l_max 0 / 1 widths, a two-layer full-O(3) blob and the
full-O(3) passes of three- and four-layer models."""
import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from oracle.model import OracleModel
from tests.conftest import energy_scale

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])
TOL = 1e-5


def _blob(name):
    cfg = synth.TINY if name.startswith("tiny") else synth.MAIN
    seed = 43 if name.endswith("teacher") else 42
    return cfg, synth.make_blob(cfg, seed, sigma=energy_scale(name))


def _gpu(ctx, pos, sp, cell, precision=al.ALLEGRO_FP32):
    N = len(pos)
    p = torch.tensor(pos, device="cuda")
    s = torch.tensor(sp, device="cuda", dtype=torch.int32)
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    Ei = torch.empty(N, dtype=torch.float64, device="cuda")
    E = al.allegro_energy_forces(ctx, p, s, cell, F, Ei, precision)
    return E, F.cpu().numpy().astype(np.float64), Ei.cpu().numpy()


def _compare(E, F, Ei, Er, Fr, Eir, tol=TOL):
    N = len(Fr)
    rms_ei = np.sqrt(np.mean(Eir ** 2))
    if abs(Er) >= 1e-3 * N:
        assert abs(E - Er) <= tol * abs(Er), (E, Er)
    else:
        assert abs(E - Er) <= tol * N * rms_ei, (E, Er)
    assert np.abs(Ei - Eir).max() <= tol * max(rms_ei, 1e-12)
    err = np.abs(F - Fr).max() / np.abs(Fr).max()
    assert err <= tol, err


@pytest.fixture(scope="module")
def tiny():
    cfg, blob = _blob("tiny")
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    yield ctx, OracleModel(blob)
    al.allegro_destroy(ctx)


@pytest.fixture(scope="module")
def main():
    cfg, blob = _blob("main")
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    yield ctx, OracleModel(blob)
    al.allegro_destroy(ctx)


def test_tiny_64_atoms(tiny):
    ctx, orc = tiny
    pos, sp, cell = synth.make_ammonia(16, 0)
    E, F, Ei = _gpu(ctx, pos, sp, cell)
    Er, Fr, Eir, _ = orc.energy_forces(pos, sp, np.diag(cell))
    _compare(E, F, Ei, Er, Fr, Eir)


@pytest.mark.parametrize("n_mol,seed", [(16, 3), (108, 5), (250, 9)])
def test_main_small_systems(main, n_mol, seed):
    """64 atoms (several images per partner, rc > L/2), 432 (3 cells), 1000."""
    ctx, orc = main
    pos, sp, cell = synth.make_ammonia(n_mol, seed)
    E, F, Ei = _gpu(ctx, pos, sp, cell)
    Er, Fr, Eir, _ = orc.energy_forces(pos, sp, np.diag(cell))
    _compare(E, F, Ei, Er, Fr, Eir)


@pytest.mark.parametrize("l_max", [0, 1])
@pytest.mark.parametrize("n_mol,seed", [(108, 5), (250, 9)])
def test_lmax_sweep_models(l_max, n_mol, seed):
    """The main model's widths at l_max 0 and 1 (Table 2's l_max sweep):
    432 and 1,000 atoms against the oracle of the same model."""
    cfg = synth.ModelConfig(r_cut=synth.MAIN.r_cut, l_max=l_max, n_layers=synth.MAIN.n_layers,
                            n_channels=synth.MAIN.n_channels, latent=synth.MAIN.latent,
                            energy=synth.MAIN.energy, avg_num_neighbors=synth.MAIN.avg_num_neighbors)
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(n_mol, seed)
    E, F, Ei = _gpu(ctx, pos, sp, cell)
    Er, Fr, Eir, _ = OracleModel(blob).energy_forces(pos, sp, np.diag(cell))
    _compare(E, F, Ei, Er, Fr, Eir)
    al.allegro_destroy(ctx)


def test_main_6912(main):
    ctx, orc = main
    pos, sp, cell = synth.make_ammonia(1728, 0)
    E, F, Ei = _gpu(ctx, pos, sp, cell)
    Er, Fr, Eir, _ = orc.energy_forces(pos, sp, np.diag(cell))
    _compare(E, F, Ei, Er, Fr, Eir)
    assert abs(np.sqrt(np.mean(Fr ** 2)) - 1.0) < 1e-6          # calibrated force scale


def test_host_buffers_and_determinism(main):
    ctx, orc = main
    pos, sp, cell = synth.make_ammonia(108, 2)
    N = len(pos)
    F1 = np.zeros((N, 3), np.float32)
    E1 = al.allegro_energy_forces(ctx, pos, sp.astype(np.int32), cell, F1, None)
    E2, F2, _ = _gpu(ctx, pos, sp, cell)
    assert E1 == E2 and np.array_equal(F1.astype(np.float64), F2)   # bitwise rerun


def test_sampled_atoms_110592(main):
    ctx, orc = main
    pos, sp, cell = synth.make_ammonia(27648, 0)
    E, F, Ei = _gpu(ctx, pos, sp, cell)
    rng = np.random.default_rng(1)
    fmax = 0.0
    errs = []
    for k in rng.choice(len(pos), 12, replace=False):
        ek, fk = orc.local_energy_force(pos, sp, np.diag(cell), int(k))
        errs.append(np.abs(F[k] - fk).max())
        fmax = max(fmax, np.abs(fk).max())
        assert abs(Ei[k] - ek) <= 1e-5 * max(1.0, abs(ek)) + 1e-6
    assert max(errs) <= 1e-5 * max(fmax, 1.0)
    assert np.abs(F.sum(0)).max() <= 1e-3 * np.sqrt(len(pos))   # net force ~ 0


def test_invalid_inputs(main):
    ctx, _ = main
    pos, sp, cell = synth.make_ammonia(16, 0)
    bad = sp.copy().astype(np.int32)
    bad[3] = 7
    with pytest.raises(al.AllegroError) as e:
        al.allegro_energy_forces(ctx, pos, bad, cell)
    assert e.value.code == 1
    tri = cell.copy()
    tri[0, 1] = 0.5
    with pytest.raises(al.AllegroError) as e:
        al.allegro_energy_forces(ctx, pos, sp.astype(np.int32), tri)
    assert e.value.code == 4
    with pytest.raises(al.AllegroError) as e:
        al.allegro_energy_forces(ctx, pos, sp.astype(np.int32), np.diag([2.0, 2.0, 2.0]))
    assert e.value.code == 3
    p = pos.copy()
    p[5, 1] = np.nan
    with pytest.raises(al.AllegroError) as e:
        al.allegro_energy_forces(ctx, p, sp.astype(np.int32), cell)
    assert e.value.code == 7
    # the context stays usable after each rejected call
    E, F, Ei = _gpu(ctx, pos, sp, cell)
    assert np.isfinite(E)


@pytest.mark.parametrize("precision", [al.ALLEGRO_FP32, al.ALLEGRO_FP16_SPLIT], ids=["fp32", "fp16split"])
def test_no_pairs_and_single_atom(main, precision):
    """Degenerate inputs: atoms farther apart than r_cut (an empty pair list)
    and a single atom.  E_i = mu_Z (0 here) and every force is zero, exactly,
    on both paths; a following ordinary call is unaffected."""
    ctx, orc = main
    cell = np.diag([30.0, 30.0, 30.0])
    pos = np.array([[1.0, 1.0, 1.0], [8.0, 1.0, 1.0], [1.0, 9.5, 20.0]])
    sp = np.array([0, 1, 1])
    for p, s in ((pos, sp), (pos[:1], sp[:1])):
        E, F, Ei = _gpu(ctx, p, s, cell, precision)
        Er, Fr, Eir, pairs = orc.energy_forces(p, s, np.diag(cell))
        assert len(pairs[0]) == 0 and al.allegro_query(ctx, al.ALLEGRO_Q_N_PAIRS) == 0
        assert E == Er and np.array_equal(Ei, Eir) and not np.any(F) and not np.any(Fr)
    p2, s2, c2 = synth.make_ammonia(16, 3)
    E, F, Ei = _gpu(ctx, p2, s2, c2)
    Er, Fr, Eir, _ = orc.energy_forces(p2, s2, np.diag(c2))
    _compare(E, F, Ei, Er, Fr, Eir)


def test_full_o3_two_layer_blob():
    """A full-O(3) blob (parity flag 1: pseudotensor mixing matrices for the
    odd paths of layer 1) of the 2-layer main model, against the oracle's
    full-O(3) evaluation, which forms the odd paths and pseudotensors: the
    FP32 passes at 1e-5 and the split tensor-core mode within 2e-3 eV/A.
    (With two layers the odd paths cannot reach the energy, which the oracle's
    own pins show; the library builds the natural-parity passes.)"""
    import dataclasses
    cfg = dataclasses.replace(synth.MAIN, parity=1)
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    orc = OracleModel(blob)
    assert orc.o3 and "layer1.mix1p" in orc.w
    pos, sp, cell = synth.make_ammonia(108, 5)
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    try:
        E, F, Ei = _gpu(ctx, pos, sp, cell)
        Es, Fs, _ = _gpu(ctx, pos, sp, cell, al.ALLEGRO_FP16_SPLIT)
    finally:
        al.allegro_destroy(ctx)
    Er, Fr, Eir, _ = orc.energy_forces(pos, sp, np.diag(cell))
    _compare(E, F, Ei, Er, Fr, Eir)
    assert np.abs(Fs - Fr).max() <= 2e-3


def _o3_pair(base, l_max, n_layers):
    """(cfg, natural blob, full-O(3) blob) sharing the natural-parity model;
    the pseudotensor weights scaled up (layer-1 pseudotensor mixing x100, the
    pseudotensor-input columns of later mixings x30) so that the odd paths,
    which reach the energy only through a second-order chain and weakly for
    these synthetic weights, move the forces by ~5e-3 of max |F|."""
    import dataclasses
    from tests.test_oracle_o3 import _blobs
    cfg = dataclasses.replace(synth.TINY if base == "tiny" else synth.MAIN, l_max=l_max, n_layers=n_layers)
    nat, o3 = _blobs(cfg, 42, pseudo_scale=100.0, cross_scale=30.0)
    return cfg, nat, o3


@pytest.mark.parametrize("base,l_max,n_layers", [("tiny", 1, 3), ("tiny", 1, 4), ("main", 1, 3),
                                                 ("main", 2, 3), ("main", 2, 4)])
def test_full_o3_deep_models(base, l_max, n_layers):
    """Full-O(3) models of three and four layers run the full-O(3) FP32 passes
    (both parities per channel, every even and odd coupling path, one mixing
    block per output irrep; with four layers also the pseudoscalars of layer 2
    as inputs of layer 3).  Against the oracle's full-O(3) evaluation at the
    FP32 bounds (1e-5); and the change from the natural-parity model with the
    same shared weights (run by the natural passes) must match the oracle's
    change to 1e-2 of its size (each evaluation rounds to ~1e-6 of max |F|):
    the odd paths themselves, not only the shared part, are checked."""
    cfg, nat, o3 = _o3_pair(base, l_max, n_layers)
    pos, sp, cell = synth.make_ammonia(108, 5)
    got, ref = {}, {}
    for key, blob in (("nat", nat), ("o3", o3)):
        ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
        try:
            got[key] = _gpu(ctx, pos, sp, cell)
        finally:
            al.allegro_destroy(ctx)
        ref[key] = OracleModel(blob).energy_forces(pos, sp, np.diag(cell))[:3]
        _compare(*got[key], *ref[key])
    dF, dFr = got["o3"][1] - got["nat"][1], ref["o3"][1] - ref["nat"][1]
    dEi, dEir = got["o3"][2] - got["nat"][2], ref["o3"][2] - ref["nat"][2]
    assert np.abs(dFr).max() >= 1e-3 * np.abs(ref["nat"][1]).max()       # the odd paths are active
    assert np.abs(dF - dFr).max() <= 1e-2 * np.abs(dFr).max()
    assert np.abs(dEi - dEir).max() <= 1e-2 * np.abs(dEir).max()


def test_full_o3_nve_trajectory_and_weights():
    """Twenty FP32 NVE steps of the 3-layer full-O(3) main model on 432 atoms
    against the oracle's trajectory (bounds of the FP32 trajectory test); then
    the weight vector: get_weights returns the blob's tensors in blob order
    (pseudotensor mixing matrices after the natural ones of each layer), and
    set_weights with layer 1's pseudotensor mixing zeroed gives the oracle's
    energy of that model (the device blocks are filled through the same path
    map as at creation)."""
    from oracle.md import velocity_verlet
    cfg, _, o3 = _o3_pair("main", 2, 3)
    orc = OracleModel(o3)
    pos, sp, cell = synth.make_ammonia(108, 5)
    L = np.diag(cell)
    v0 = synth.make_velocities(sp, 200.0, 1)
    n = 20
    ctx = al.allegro_create(o3, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    try:
        al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
        en = np.zeros((n, 3))
        al.allegro_md_step_nve(ctx, 0.5, n, None, en)
        P, V = np.zeros_like(pos), np.zeros_like(pos)
        assert al.allegro_md_get_state(ctx, P, V) == n
        nw = al.allegro_query(ctx, al.ALLEGRO_Q_N_PARAMS)
        wv = np.zeros(nw, np.float32)
        al.allegro_get_weights(ctx, wv)
        offs, o = {}, 0
        for name in orc.names:
            offs[name] = (o, orc.w[name].numel())
            o += orc.w[name].numel()
        assert o == nw
        for name in ("layer1.mix1p", "layer2.mix2p", "layer2.mix0"):
            a, m = offs[name]
            np.testing.assert_array_equal(wv[a:a + m], orc.w[name].numpy().ravel().astype(np.float32))
        w2 = wv.copy()
        for name in orc.names:
            if name.startswith("layer1.") and name.endswith("p"):
                a, m = offs[name]
                w2[a:a + m] = 0.0
                orc.w[name] = orc.w[name] * 0.0
        al.allegro_set_weights(ctx, w2)
        E, F, Ei = _gpu(ctx, pos, sp, cell)
    finally:
        al.allegro_destroy(ctx)
    ref = velocity_verlet(lambda p: OracleModel(o3).energy_forces(p, sp, L)[:2], pos, v0, MASS[sp], L, 0.5, n)
    d = P - ref["pos"]
    d -= np.round(d / L) * L
    assert np.abs(d).max() < 1e-5
    assert np.abs(V - ref["vel"]).max() < 1e-5
    np.testing.assert_allclose(en[:, 0], ref["epot"], rtol=0, atol=1e-4 * abs(ref["epot"]).max())
    Er, Fr, Eir, _ = orc.energy_forces(pos, sp, L)
    _compare(E, F, Ei, Er, Fr, Eir)


def _waves(v):
    return [(v >> (4 * q)) & 15 for q in range(5)]


def test_launch_shape_autotuner_keeps_the_bits():
    """The FP32 passes take their launch shapes (waves of one block per SM,
    per pass) from the autotuner, tuned on the first evaluation of a
    context.  A context tuned and sized on the 110,592-atom system and one
    tuned on the 432-atom system launch the 432-atom evaluation with
    different grids; energies, per-atom energies and forces must agree
    bitwise (every tile's work and partial rows are fixed by the tile)."""
    cfg, blob = _blob("main")
    pos, sp, cell = synth.make_ammonia(108, 2)
    bpos, bsp, bcell = synth.make_ammonia(27648, 0)
    ctx2 = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    try:
        _gpu(ctx2, bpos, bsp, bcell)
        E2, F2, Ei2 = _gpu(ctx2, pos, sp, cell)
        w2 = al.allegro_query(ctx2, al.ALLEGRO_Q_FP32_LAUNCH)
    finally:
        al.allegro_destroy(ctx2)
    ctx1 = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    try:
        E1, F1, Ei1 = _gpu(ctx1, pos, sp, cell)
        w1 = al.allegro_query(ctx1, al.ALLEGRO_Q_FP32_LAUNCH)
    finally:
        al.allegro_destroy(ctx1)
    print("tuned waves (A, B, C, B^T, A^T):", _waves(w1), _waves(w2))
    for w in (w1, w2):
        assert all(x in (1, 2, 4, 8) for x in _waves(w))
    assert E1 == E2 and np.array_equal(F1, F2) and np.array_equal(Ei1, Ei2)
