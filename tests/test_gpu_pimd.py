"""GPU ring-polymer MD (Sec. 6, Fig. 6) vs the oracle: the replicas' energies
and forces come from one pass sequence over all replicas, the ring springs
are propagated exactly in normal modes."""
import numpy as np
import pytest
import torch

import synth
import paper_2303_08169_gb300 as al
from oracle.md import kinetic_energy
from oracle.model import OracleModel
from oracle.pimd import omega_p, rpmd, spring_energy
from tests.conftest import energy_scale

pytestmark = pytest.mark.gpu
MASS = np.array([14.007, 1.008])


def _ring(pos, sp, P, T, seed):
    """P replicas around pos (0.03 A Gaussian offsets, unwrapped) with
    Maxwell velocities at T per replica."""
    rng = np.random.default_rng(seed)
    q = pos[None] + 0.03 * rng.normal(size=(P,) + pos.shape)
    v = np.stack([synth.make_velocities(sp, T, seed + 1 + k) for k in range(P)])
    return q, v


def test_tiny_pimd_matches_oracle_trajectory():
    """Four replicas of 64 atoms at 200 K, 20 steps of 0.5 fs: bead positions
    and velocities, the mean replica energy, the kinetic energy and H_P
    follow the oracle's ring-polymer integrator."""
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    orc = OracleModel(blob)
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    P, T, n = 4, 200.0, 20
    q0, v0 = _ring(pos, sp, P, T, 3)
    al.allegro_pimd_init(ctx, q0, v0, sp.astype(np.int32), cell, T)
    en = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    al.allegro_pimd_step(ctx, 0.5, n, en)
    Q = np.zeros_like(q0)
    V = np.zeros_like(v0)
    al.allegro_pimd_get_state(ctx, Q, V)
    ref = rpmd(lambda p: orc.energy_forces(p, sp, L)[:2], q0, v0, MASS[sp], 0.5, n, T)
    en = en.cpu().numpy()
    # springs move the beads by far more than the FP32 force error
    assert np.abs(ref["q"] - q0 - 0.5 * n * v0).max() > 1e-3
    assert np.abs(Q - ref["q"]).max() < 1e-5
    assert np.abs(V - ref["v"]).max() < 1e-5
    scale = abs(ref["vmean"]).max()
    np.testing.assert_allclose(en[:, 0], ref["vmean"], rtol=0, atol=1e-4 * scale)
    np.testing.assert_allclose(en[:, 1], ref["ekin"], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(en[:, 2], ref["hp"], rtol=0, atol=1e-4 * scale)
    m = MASS[sp]
    ek = sum(kinetic_energy(V[k], m) for k in range(P))
    assert abs(ek - en[-1, 1]) < 1e-9 * en[-1, 1]
    hp = ek + spring_energy(Q, m, omega_p(P, T)) + P * en[-1, 0]
    assert abs(hp - en[-1, 2]) < 1e-9 * abs(hp) + 1e-9
    al.allegro_destroy(ctx)


def test_single_replica_is_nve():
    """P = 1 has no springs: the steps are the NVE velocity-Verlet steps
    (positions agree up to the periodic wrap the NVE state applies)."""
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    v0 = synth.make_velocities(sp, 200.0, 1)
    n = 20
    al.allegro_md_init(ctx, pos, v0, sp.astype(np.int32), cell)
    e_nve = np.zeros((n, 3))
    al.allegro_md_step_nve(ctx, 0.5, n, None, e_nve)
    P1 = np.zeros((len(pos), 3))
    V1 = np.zeros((len(pos), 3))
    al.allegro_md_get_state(ctx, P1, V1)
    al.allegro_pimd_init(ctx, pos[None], v0[None], sp.astype(np.int32), cell, 200.0)
    e_rp = np.zeros((n, 3))
    al.allegro_pimd_step(ctx, 0.5, n, e_rp)
    Q = np.zeros((1, len(pos), 3))
    V = np.zeros((1, len(pos), 3))
    al.allegro_pimd_get_state(ctx, Q, V)
    d = Q[0] - P1
    d -= np.round(d / L) * L
    assert np.abs(d).max() < 1e-8
    assert np.abs(V[0] - V1).max() < 1e-8
    scale = abs(e_nve[:, 0]).max()
    np.testing.assert_allclose(e_rp[:, 0], e_nve[:, 0], rtol=0, atol=1e-6 * scale)
    np.testing.assert_allclose(e_rp[:, 1], e_nve[:, 1], rtol=1e-8)
    np.testing.assert_allclose(e_rp[:, 2], e_nve[:, 2], rtol=0, atol=1e-6 * scale)
    al.allegro_destroy(ctx)


@pytest.mark.parametrize("precision", [al.ALLEGRO_FP32, al.ALLEGRO_BF16, al.ALLEGRO_FP16_SPLIT])
def test_batched_replicas_match_single_evaluations(precision):
    """Six replicas of the 6,912-atom system in one pass sequence (replica
    pair ranges start mid-tile): the mean replica energy equals the mean of
    the replicas evaluated one by one at the same precision."""
    cfg = synth.MAIN
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("main"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(1728, 0)
    P, T = 6, 200.0
    q0, v0 = _ring(pos, sp, P, T, 5)
    sp32 = sp.astype(np.int32)
    al.allegro_set_md_precision(ctx, precision)
    al.allegro_pimd_init(ctx, q0, v0, sp32, cell, T)
    en = np.zeros((1, 3))
    al.allegro_pimd_step(ctx, 0.25, 1, en)
    Q = np.zeros_like(q0)
    V = np.zeros_like(v0)
    al.allegro_pimd_get_state(ctx, Q, V)
    e_one = [al.allegro_energy_forces(ctx, Q[k], sp32, cell, precision=precision) for k in range(P)]
    assert abs(np.mean(e_one) - en[0, 0]) <= 1e-5 * abs(en[0, 0])
    # the replicas differ: their energies are not one number
    assert np.ptp(e_one) > 1e-6
    al.allegro_destroy(ctx)


def test_pimd_conserves_hp_and_resumes():
    """200 steps: H_P stays within a small fraction of the kinetic-energy
    swing, and two calls of 100 steps equal one call of 200 (bitwise: the
    pass sequence is deterministic), also with an energy evaluation of a
    larger system in between (the ring state lives in its own arrays; the
    shared buffers grow and the step graph is captured again)."""
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    P, T = 8, 200.0
    q0, v0 = _ring(pos, sp, P, T, 7)
    sp32 = sp.astype(np.int32)
    al.allegro_pimd_init(ctx, q0, v0, sp32, cell, T)
    e1 = np.zeros((200, 3))
    al.allegro_pimd_step(ctx, 0.25, 200, e1)
    al.allegro_pimd_init(ctx, q0, v0, sp32, cell, T)
    a, b = np.zeros((100, 3)), np.zeros((100, 3))
    al.allegro_pimd_step(ctx, 0.25, 100, a)
    big, sbig, cbig = synth.make_ammonia(250, 4)
    al.allegro_energy_forces(ctx, big, sbig.astype(np.int32), cbig)
    al.allegro_pimd_step(ctx, 0.25, 100, b)
    assert np.array_equal(np.vstack([a, b]), e1)
    dH = np.abs(e1[:, 2] - e1[0, 2]).max()
    dK = np.ptp(e1[:, 1])
    assert dK > 0 and dH < 0.05 * dK
    al.allegro_destroy(ctx)


def test_shared_buffer_calls_end_the_md_state():
    """allegro_energy_forces and the ring-polymer calls reuse the MD state's
    buffers: the next NVE step asks for allegro_md_init instead of stepping
    a clobbered state."""
    cfg = synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=energy_scale("tiny"))
    ctx = al.allegro_create(blob, MASS, cfg.r_cut, cfg.l_max, cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(16, 0)
    sp32 = sp.astype(np.int32)
    v0 = synth.make_velocities(sp, 200.0, 1)
    al.allegro_md_init(ctx, pos, v0, sp32, cell)
    al.allegro_md_step_nve(ctx, 0.5, 2)
    al.allegro_energy_forces(ctx, pos, sp32, cell)
    with pytest.raises(al.AllegroError):
        al.allegro_md_step_nve(ctx, 0.5, 2)
    al.allegro_md_init(ctx, pos, v0, sp32, cell)
    al.allegro_md_step_nve(ctx, 0.5, 2)
    q0, v = _ring(pos, sp, 2, 200.0, 9)
    al.allegro_pimd_init(ctx, q0, v, sp32, cell, 200.0)
    with pytest.raises(al.AllegroError):
        al.allegro_md_step_nvt(ctx, 0.5, 2, 200.0, 10.0)
    al.allegro_pimd_step(ctx, 0.5, 2)
    assert al.allegro_query(ctx, al.ALLEGRO_Q_RP_STEP_KERNELS) > 10
    al.allegro_destroy(ctx)


@pytest.mark.parametrize("cfg_name,n_mol,P", [("tiny", 16, 3), ("main", 108, 4)])
def test_ring_neighbour_list_is_each_replicas_list(cfg_name, n_mol, P):
    """The ring's one neighbour build (small-box mode at 64 atoms, cell mode at
    432) is, bit for bit, each replica's own pair list (the oracle's canonical
    order) with atom indices offset by k n, and its reverse index maps every
    pair to (j, i, -n) inside the same replica."""
    from oracle.neighbors import pairs_bruteforce, reverse_index
    cfg = synth.TINY if cfg_name == "tiny" else synth.MAIN
    ctx = al.allegro_create(synth.make_blob(cfg, 42, sigma=energy_scale(cfg_name)), MASS, cfg.r_cut, cfg.l_max,
                            cfg.n_layers)
    pos, sp, cell = synth.make_ammonia(n_mol, 2)
    L = np.diag(cell)
    n = len(pos)
    q0, v0 = _ring(pos, sp, P, 200.0, 13)
    q0[1] += L                                          # a replica shifted by a whole box: same list
    al.allegro_pimd_init(ctx, q0, v0, sp.astype(np.int32), cell, 200.0)
    n_pairs = al.allegro_query(ctx, al.ALLEGRO_Q_N_PAIRS)
    row = np.zeros(P * n + 1, np.int32)
    col = np.zeros(n_pairs, np.int32)
    img = np.zeros((n_pairs, 3), np.int8)
    rev = np.zeros(n_pairs, np.int32)
    al.allegro_get_neighbors(ctx, row, col, img, rev)
    gi = np.repeat(np.arange(P * n), np.diff(row.astype(np.int64)))
    RI, RJ, RN, RR = [], [], [], []
    off = 0
    for k in range(P):
        ri, rj, rn = pairs_bruteforce(q0[k], L, cfg.r_cut)
        RI.append(ri + k * n)
        RJ.append(rj + k * n)
        RN.append(rn)
        RR.append(reverse_index(ri, rj, rn, n) + off)
        off += len(ri)
    assert n_pairs == off
    assert np.array_equal(gi, np.concatenate(RI))
    assert np.array_equal(col.astype(np.int64), np.concatenate(RJ))
    assert np.array_equal(img.astype(np.int64), np.concatenate(RN))
    assert np.array_equal(rev.astype(np.int64), np.concatenate(RR))
    al.allegro_destroy(ctx)
