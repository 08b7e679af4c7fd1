"""Pins for the oracle's energy model and forces.

The paper fixes E = sum of pair energies within a cutoff, E(3) equivariance
(Sec. 2.1) and f = -dE/dr (Eq. 1); these tests check the oracle against a
dimer closed form, O(3)/translation/permutation invariance, zero net force,
central finite differences, smoothness at r_cut and locality.
"""
import math

import numpy as np
import pytest
import torch
from sympy.physics.quantum.cg import CG

import synth
from oracle.model import OracleModel
from oracle.neighbors import pairs_bruteforce
from oracle.sph import coupling_paths

MINI = synth.ModelConfig(r_cut=4.5, l_max=2, n_layers=2, n_channels=4,
                         latent=(8, 8), energy=(8,), avg_num_neighbors=7.0,
                         sigma=(1.3, 0.7), mu=(0.25, -0.5))
BIG = np.array([60.0, 60.0, 60.0])


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _lin(W, x):
    return W @ x / math.sqrt(W.shape[1])


def dimer_energy(cfg, W, d, sA, sB):
    """Closed form for two atoms: every tensor is (radial) x Y_l(u), and the
    coupling of Y_l1(u) with Y_l2(u) along a path is kappa Y_l3(u) with
    kappa = sqrt((2l1+1)(2l2+1)) |<l1 0 l2 0|l3 0>| / (2l3+1) (sympy CG)."""
    rc, S, C, lmax, nu = cfg.r_cut, cfg.n_species, cfg.n_channels, cfg.l_max, cfg.avg_num_neighbors
    paths = coupling_paths(lmax)
    kappa = {p: math.sqrt((2 * p[0] + 1) * (2 * p[1] + 1)) * abs(float(CG(p[0], 0, p[1], 0, p[2], 0).doit())) / (2 * p[2] + 1)
             for p in paths}
    x_ = d / rc
    fc = 1 - 28 * x_ ** 6 + 48 * x_ ** 7 - 21 * x_ ** 8
    B = np.array([math.sqrt(2 / rc) * math.sin(k * math.pi * d / rc) / d for k in range(1, cfg.n_bessel + 1)])
    nlat = len(cfg.latent)

    def pair(si, sj):
        h = np.concatenate([np.eye(S)[si], np.eye(S)[sj], B])
        a = h
        for k in range(nlat):
            a = _silu(_lin(W[f"twobody.{k}"], a))
        x = fc * a
        rad = _lin(W["embed"], x).reshape(C, lmax + 1)       # radial part of V
        for layer in range(1, cfg.n_layers + 1):
            e = _lin(W[f"layer{layer}.env"], x) / math.sqrt(nu)
            T = {p: rad[:, p[0]] * e * kappa[p] for p in paths}  # radial part of T
            sc = [p for p in paths if p[2] == 0]
            s = np.stack([T[p] for p in sc], 1).reshape(-1)
            if layer < cfg.n_layers:
                new = np.zeros((C, lmax + 1))
                for l3 in range(lmax + 1):
                    ps = [p for p in paths if p[2] == l3]
                    t = np.stack([T[p] for p in ps], 1).reshape(-1)
                    new[:, l3] = W[f"layer{layer}.mix{l3}"] @ t / math.sqrt(C * len(ps))
                rad = new
            a = np.concatenate([x, s])
            for k in range(nlat):
                a = _silu(_lin(W[f"layer{layer}.latent.{k}"], a))
            x = (x + fc * a) / math.sqrt(2)
        a = x
        for k in range(len(cfg.energy)):
            a = _silu(_lin(W[f"energy.{k}"], a))
        return float(_lin(W["energy.out"], a)[0])

    return (cfg.sigma[sA] * pair(sA, sB) + cfg.mu[sA]
            + cfg.sigma[sB] * pair(sB, sA) + cfg.mu[sB])


MINI_L0 = synth.ModelConfig(r_cut=4.5, l_max=0, n_layers=2, n_channels=4, latent=(8, 8), energy=(8,),
                            avg_num_neighbors=7.0, sigma=(1.3, 0.7), mu=(0.25, -0.5))
MINI_L1 = synth.ModelConfig(r_cut=4.5, l_max=1, n_layers=3, n_channels=4, latent=(8, 8), energy=(8,),
                            avg_num_neighbors=7.0, sigma=(1.3, 0.7), mu=(0.25, -0.5))


@pytest.mark.parametrize("cfg", [MINI, MINI_L0, MINI_L1, synth.TINY.with_sigma(1.7)],
                         ids=["mini_l2_2layers", "mini_l0_2layers", "mini_l1_3layers", "tiny"])
def test_dimer_closed_form(cfg):
    W = synth.make_weights(cfg, 11)
    model = OracleModel(synth.write_blob(cfg, W))
    rng = np.random.default_rng(0)
    for d in (0.9, 1.7, 2.6, 3.8):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.array([[30.0, 30.0, 30.0], [30.0, 30.0, 30.0]]) + np.array([[0, 0, 0], d * u])
        E, F, Ei, _ = model.energy_forces(pos, np.array([0, 1]), BIG)
        ref = dimer_energy(cfg, W, d, 0, 1)
        assert abs(E - ref) <= 1e-12 * max(1.0, abs(ref))


def _cluster(n_mol=6, seed=2):
    pos, sp, _ = synth.make_ammonia(n_mol, seed)
    return pos - pos.mean(0) + 30.0, sp


def _rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("cfg", [MINI, MINI_L1], ids=["l2", "l1"])
def test_o3_invariance_and_force_covariance(cfg):
    model = OracleModel(synth.make_blob(cfg, 5))
    pos, sp = _cluster()
    E0, F0, _, _ = model.energy_forces(pos, sp, BIG)
    rng = np.random.default_rng(1)
    for k in range(100):
        R = _rot(rng) * (-1 if k % 2 else 1)
        p = (pos - 30.0) @ R.T + 30.0
        E, F, _, _ = model.energy_forces(p, sp, BIG)
        assert abs(E - E0) <= 1e-12 * max(1, abs(E0))
        np.testing.assert_allclose(F, F0 @ R.T, atol=1e-11 * np.abs(F0).max())


def test_periodic_symmetries_translation_permutation(tiny_model):
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    E0, F0, Ei0, _ = tiny_model.energy_forces(pos, sp, L)
    rng = np.random.default_rng(2)
    for _ in range(5):                           # translations
        E, F, _, _ = tiny_model.energy_forces(pos + rng.uniform(-20, 20, size=3), sp, L)
        assert abs(E - E0) <= 1e-12 * abs(E0)
        np.testing.assert_allclose(F, F0, atol=1e-11)
    for _ in range(3):                           # cube symmetries (axis permutation + reflection)
        perm = rng.permutation(3)
        sign = rng.choice([-1.0, 1.0], size=3)
        p = pos[:, perm] * sign[None, :]
        E, F, _, _ = tiny_model.energy_forces(p, sp, L)
        assert abs(E - E0) <= 1e-12 * abs(E0)
        np.testing.assert_allclose(F, F0[:, perm] * sign[None, :], atol=1e-11)
    # same-species permutation
    order = np.arange(len(sp))
    H = np.nonzero(sp == 1)[0]
    order[H] = rng.permutation(H)
    E, F, Ei, _ = tiny_model.energy_forces(pos[order], sp[order], L)
    assert abs(E - E0) <= 1e-12 * abs(E0)
    np.testing.assert_allclose(F, F0[order], atol=1e-11)
    np.testing.assert_allclose(Ei, Ei0[order], atol=1e-12)


def test_zero_net_force_and_finite_differences(tiny_model):
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    E0, F0, _, _ = tiny_model.energy_forces(pos, sp, L)
    assert np.abs(F0.sum(0)).max() <= 1e-10 * np.abs(F0).max() * len(pos)
    h = 1e-4
    rng = np.random.default_rng(3)
    for _ in range(12):
        a, c = int(rng.integers(len(pos))), int(rng.integers(3))
        p1, p2 = pos.copy(), pos.copy()
        p1[a, c] += h
        p2[a, c] -= h
        fd = -(tiny_model.energy_forces(p1, sp, L)[0] - tiny_model.energy_forces(p2, sp, L)[0]) / (2 * h)
        assert abs(fd - F0[a, c]) <= 1e-6 * np.abs(F0).max()


def test_smooth_at_cutoff():
    cfg = synth.TINY.with_sigma(1.0)
    model = OracleModel(synth.make_blob(cfg, 3))
    rc = cfg.r_cut
    vals = []
    for d in (rc - 1e-3, rc - 1e-6, rc + 1e-6):
        pos = np.array([[30.0, 30.0, 30.0], [30.0 + d, 30.0, 30.0]])
        E, F, _, _ = model.energy_forces(pos, np.array([0, 1]), BIG)
        vals.append((E - sum(cfg.mu), np.abs(F).max()))
    assert abs(vals[2][0]) == 0 and vals[2][1] == 0
    assert abs(vals[1][0]) < 1e-12 and vals[1][1] < 1e-9      # O(delta^3) and O(delta^2)
    assert abs(vals[0][0]) < 1e-4


def test_locality(tiny_model):
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell) * 2.0                       # dilute box so far atoms exist
    _, _, Ei0, _ = tiny_model.energy_forces(pos, sp, L)
    i0 = 0
    d = pos - pos[i0]
    dist = np.sqrt((d * d).sum(1))
    far = int(np.argmax(dist))
    assert dist[far] > tiny_model.rc + 0.5
    p = pos.copy()
    p[far] += 0.1 * (p[far] - pos[i0]) / dist[far]   # moves further away
    _, _, Ei, _ = tiny_model.energy_forces(p, sp, L)
    assert Ei[i0] == Ei0[i0]


def test_local_evaluation_matches_full():
    model = OracleModel(synth.make_blob(synth.TINY.with_sigma(2.0), 42))
    pos, sp, cell = synth.make_ammonia(250, 4)     # L = 21.9 > 4 rc + 1
    L = np.diag(cell)
    E, F, Ei, _ = model.energy_forces(pos, sp, L)
    for k in (0, 123, 999):
        ek, fk = model.local_energy_force(pos, sp, L, k)
        assert abs(ek - Ei[k]) <= 1e-11 * max(1, abs(Ei[k]))
        np.testing.assert_allclose(fk, F[k], atol=1e-10 * np.abs(F).max())
