"""Pins for the oracle's ring-polymer MD (Sec. 6, Fig. 6)."""
import math

import numpy as np

from oracle.md import KAPPA, velocity_verlet
from oracle.pimd import free_ring_step, normal_modes, omega_p, rpmd, spring_energy


def test_normal_modes_diagonalise_the_ring():
    """C is orthogonal and turns the ring's spring matrix (2 on the diagonal,
    -1 to each neighbour, cyclic) into diag((omega_k / omega_P)^2)."""
    for P in (1, 2, 5, 8, 32):
        C, w = normal_modes(P)
        assert np.allclose(C.T @ C, np.eye(P), atol=1e-13)
        A = 2.0 * np.eye(P) - np.roll(np.eye(P), 1, axis=1) - np.roll(np.eye(P), -1, axis=1)
        if P == 1:
            A = np.zeros((1, 1))
        if P == 2:
            A = np.array([[2.0, -2.0], [-2.0, 2.0]])
        assert np.allclose(C.T @ A @ C, np.diag(w * w), atol=1e-12)


def test_free_ring_polymer_exact():
    """Without physical forces the propagation is exact: K + spring energy is
    conserved, the centroid moves in a straight line, and it matches the
    closed-form evolution of each normal mode after many small or one large
    step."""
    rng = np.random.default_rng(0)
    P, N = 8, 5
    m = np.array([14.007, 1.008, 1.008, 1.008, 14.007])
    q = rng.normal(size=(P, N, 3)) * 0.05 + rng.normal(size=(1, N, 3))
    v = rng.normal(size=(P, N, 3)) * 0.01
    wp = omega_p(P, 200.0)

    def energy(qq, vv):
        return 0.5 * float((m[None, :, None] * vv * vv).sum()) / KAPPA + spring_energy(qq, m, wp)

    e0 = energy(q, v)
    qa, va = q.copy(), v.copy()
    for _ in range(400):
        qa, va = free_ring_step(qa, va, 0.05, wp)
    assert abs(energy(qa, va) - e0) <= 1e-11 * e0
    np.testing.assert_allclose(qa.mean(axis=0), q.mean(axis=0) + 20.0 * v.mean(axis=0), atol=1e-12)
    qb, vb = free_ring_step(q, v, 20.0, wp)
    np.testing.assert_allclose(qa, qb, atol=1e-9)
    np.testing.assert_allclose(va, vb, atol=1e-10)


def test_single_replica_is_verlet():
    """P = 1: no springs, the steps are velocity Verlet."""
    rng = np.random.default_rng(1)
    ctr = 100.0 + 10.0 * rng.random((6, 3))
    q0 = ctr + 0.2 * rng.normal(size=(6, 3))
    v0 = 0.01 * rng.normal(size=(6, 3))
    m = np.full(6, 14.007)

    def ffn(p):
        d = p - ctr
        return 0.5 * 2.0 * float((d * d).sum()), -2.0 * d

    a = rpmd(ffn, q0[None], v0[None], m, 0.5, 40, 200.0)
    b = velocity_verlet(ffn, q0, v0, m, np.array([1000.0] * 3), 0.5, 40)
    assert np.abs(a["q"][0] - b["pos"]).max() < 1e-12 and np.abs(a["v"][0] - b["vel"]).max() < 1e-13
    np.testing.assert_allclose(a["hp"], b["etot"], rtol=1e-13)


def test_ring_polymer_energy_second_order():
    """With a physical potential H_P is conserved up to the splitting error,
    which shrinks about 4x when dt halves."""
    rng = np.random.default_rng(2)
    P, N = 4, 6
    ctr = 100.0 + 10.0 * rng.random((N, 3))
    m = np.where(rng.random(N) < 0.5, 14.007, 1.008)
    q0 = ctr[None] + 0.2 * rng.normal(size=(P, N, 3))
    v0 = 0.01 * rng.normal(size=(P, N, 3))

    def ffn(p):
        d = p - ctr
        r2 = (d * d).sum(axis=1, keepdims=True)
        return float((r2 + 0.25 * r2 * r2).sum()), -(2.0 + r2) * d

    dev = []
    for dt, n in ((0.2, 100), (0.1, 200)):
        o = rpmd(ffn, q0, v0, m, dt, n, 300.0)
        dev.append(np.abs(o["hp"] - o["hp"][0]).max())
    assert 3.0 < dev[0] / dev[1] < 5.0


def test_harmonic_ring_against_matrix_exponential():
    """Beads of atoms in harmonic wells (V = k |q - c|^2 / 2 per replica):
    the ring-polymer equations are linear, q'' = -(kappa k / m + omega_P^2 K) q
    with K the cyclic spring matrix, and their exact flow is the matrix
    exponential of the first-order system (no normal modes involved).  The
    integrator follows it with a second-order error."""
    from scipy.linalg import expm
    rng = np.random.default_rng(5)
    P, N, T, t_end = 5, 3, 300.0, 12.0
    m = np.array([14.007, 1.008, 1.008])
    kk = np.array([2.0, 0.5, 0.8])                   # eV / A^2
    c = 50.0 + 5.0 * rng.random((N, 3))
    q0 = c[None] + 0.1 * rng.normal(size=(P, N, 3))
    v0 = 0.01 * rng.normal(size=(P, N, 3))
    wp = omega_p(P, T)
    K = 2.0 * np.eye(P) - np.roll(np.eye(P), 1, axis=1) - np.roll(np.eye(P), -1, axis=1)

    def ffn(p):
        d = p - c
        return 0.5 * float((kk[:, None] * d * d).sum()), -kk[:, None] * d

    exact = np.zeros_like(q0)
    for i in range(N):
        A = KAPPA * kk[i] / m[i] * np.eye(P) + wp * wp * K
        M = np.block([[np.zeros((P, P)), np.eye(P)], [-A, np.zeros((P, P))]])
        E = expm(M * t_end)
        for a in range(3):
            y = E @ np.concatenate([q0[:, i, a] - c[i, a], v0[:, i, a]])
            exact[:, i, a] = y[:P] + c[i, a]
    err = []
    for dt in (0.1, 0.05):
        o = rpmd(ffn, q0, v0, m, dt, int(round(t_end / dt)), T)
        err.append(np.abs(o["q"] - exact).max())
    assert err[1] < 1e-4
    assert 3.5 < err[0] / err[1] < 4.5
