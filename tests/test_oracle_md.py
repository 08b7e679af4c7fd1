"""Pins for the oracle's NVE velocity Verlet (Eq. 1, Sec. 3.2), its
Nose-Hoover NVT and the >5 sigma force-outlier count (Fig. 1 caption)."""
import math

import numpy as np
import pytest

import synth
from oracle.md import KAPPA, KB_EV, kinetic_energy, nose_hoover, outlier_count, velocity_verlet


def test_verlet_harmonic_shadow_energy_exact():
    """For F = -k x, velocity Verlet conserves v^2 + w^2 (1 - w^2 dt^2 / 4) x^2
    exactly (w^2 = kappa k / m) and follows the linear map
    x' = (1 - c) x + dt v, v' = (1 - c) v - dt w^2 (1 - c/2) x, c = w^2 dt^2 / 2."""
    k, m, dt = 3.0, 2.0, 0.7
    L = np.array([1000.0, 1000.0, 1000.0])
    x0 = np.array([[500.4, 499.0, 501.3]])
    v0 = np.array([[0.01, -0.02, 0.005]])
    ctr = np.array([[500.0, 500.0, 500.0]])

    def ffn(p):
        dx = p - ctr
        return 0.5 * k * float((dx * dx).sum()), -k * dx

    out = velocity_verlet(ffn, x0, v0, np.array([m]), L, dt, 50)
    w2 = KAPPA * k / m
    c = 0.5 * w2 * dt * dt
    x, v = x0 - ctr, v0.copy()
    for _ in range(50):
        x, v = (1 - c) * x + dt * v, (1 - c) * v - dt * w2 * (1 - 0.5 * c) * x
    np.testing.assert_allclose(out["pos"] - ctr, x, atol=1e-10)
    np.testing.assert_allclose(out["vel"], v, atol=1e-12)
    q0 = (v0 ** 2).sum() + w2 * (1 - w2 * dt * dt / 4) * ((x0 - ctr) ** 2).sum()
    q1 = (out["vel"] ** 2).sum() + w2 * (1 - w2 * dt * dt / 4) * ((out["pos"] - ctr) ** 2).sum()
    assert abs(q1 - q0) <= 1e-13 * q0


def test_kinetic_energy_and_velocity_generator():
    sp = np.array([0, 1, 1, 1] * 10, dtype=np.int32)
    v = synth.make_velocities(sp, 200.0, 1)
    m = synth.MASS_AMU[sp]
    ke = kinetic_energy(v, m)
    assert abs(ke - 0.5 * (3 * 40 - 3) * 8.617333e-5 * 200.0) < 1e-12
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0, atol=1e-14)
    assert abs(kinetic_energy(np.array([[1.0, 0, 0]]), np.array([2.0])) - 1.0 / KAPPA) < 1e-12


def test_outlier_count_closed_form():
    f = np.ones((10, 3))
    assert outlier_count(f) == 0
    f[3, 1] = 100.0
    sigma = math.sqrt((29 + 1e4) / 30)       # 18.27: 100 > 5 sigma = 91.4
    assert 100 > 5 * sigma and outlier_count(f) == 1
    f[3, 1] = 80.0                           # 80 < 5 sqrt((29 + 6400)/30) = 73.2? -> yes 80 > 73.2
    assert outlier_count(f) == (1 if 80 > 5 * math.sqrt((29 + 6400) / 30) else 0)
    g = np.zeros((4, 3))
    assert outlier_count(g) == 0             # strict: 0 > 0 is false
    assert outlier_count(np.zeros((0, 3))) == 0


@pytest.mark.slow
def test_nve_drift_and_second_order(tiny_model):
    pos, sp, cell = synth.make_ammonia(16, 0)
    L = np.diag(cell)
    v0 = synth.make_velocities(sp, 200.0, 1)
    m = synth.MASS_AMU[sp]

    def ffn(p):
        E, F, _, _ = tiny_model.energy_forces(p, sp, L)
        return E, F

    kT = 8.617333e-5 * 200.0
    # seeded Gaussian weights give a stiff potential far from equilibrium at
    # the lattice start (kinetic energy rises quickly), so the absolute bound
    # is loose; the order of the integrator is the sharp check below
    a = velocity_verlet(ffn, pos, v0, m, L, 0.5, 100)
    drift = np.abs(a["etot"] - a["etot"][0]).max() / (len(sp) * kT)
    assert drift < 0.25
    # halving dt shrinks the energy fluctuation by about 4x (second order)
    b = velocity_verlet(ffn, pos, v0, m, L, 0.25, 40)
    c = velocity_verlet(ffn, pos, v0, m, L, 0.125, 80)
    fb = np.abs(b["etot"] - b["etot"][0]).max()
    fc = np.abs(c["etot"] - c["etot"][0]).max()
    assert 2.5 < fb / fc < 6.0


def _wells(n, seed=0):
    """n particles in separate anharmonic wells (no pair forces): E = sum
    k |x|^2 / 2 + a |x|^4 / 4 about fixed centres."""
    rng = np.random.default_rng(seed)
    ctr = 100.0 + 200.0 * rng.random((n, 3))
    x0 = ctr + 0.3 * rng.normal(size=(n, 3))
    v0 = 0.01 * rng.normal(size=(n, 3))
    m = np.where(rng.random(n) < 0.5, 14.007, 1.008)
    k, a = 2.0, 0.5

    def ffn(p):
        d = p - ctr
        r2 = (d * d).sum(axis=1, keepdims=True)
        return float((0.5 * k * r2 + 0.25 * a * r2 * r2).sum()), -(k + a * r2) * d

    return ffn, x0, v0, m, np.array([1000.0, 1000.0, 1000.0])


def test_nvt_without_coupling_is_verlet():
    """An infinitely heavy thermostat (tau -> inf) leaves xi at zero: the
    NVT steps are the velocity-Verlet steps."""
    ffn, x0, v0, m, L = _wells(20)
    a = nose_hoover(ffn, x0, v0, m, L, 0.5, 50, 300.0, 1e12)
    b = velocity_verlet(ffn, x0, v0, m, L, 0.5, 50)
    assert np.abs(a["pos"] - b["pos"]).max() < 1e-12 and np.abs(a["vel"] - b["vel"]).max() < 1e-13
    assert abs(a["xi"]) < 1e-15


def test_nvt_time_reversible():
    """The splitting is symmetric: n steps, then n steps with v and xi
    negated, return to the start."""
    ffn, x0, v0, m, L = _wells(20, 1)
    a = nose_hoover(ffn, x0, v0, m, L, 0.5, 200, 300.0, 20.0)
    b = nose_hoover(ffn, a["pos"], -a["vel"], m, L, 0.5, 200, 300.0, 20.0, xi=-a["xi"], eta=a["eta"])
    assert np.abs(b["pos"] - x0).max() < 1e-9
    assert np.abs(-b["vel"] - v0).max() < 1e-11
    assert abs(b["xi"]) < 1e-12


def test_nvt_extended_energy_second_order():
    """H = E_pot + K + Q xi^2 / 2 + g kT eta is conserved up to the splitting
    error, which shrinks about 4x when dt halves."""
    ffn, x0, v0, m, L = _wells(30, 2)
    dev = []
    for dt, n in ((0.4, 100), (0.2, 200)):
        o = nose_hoover(ffn, x0, v0, m, L, dt, n, 300.0, 20.0)
        dev.append(np.abs(o["hext"] - o["hext"][0]).max())
    assert 3.0 < dev[0] / dev[1] < 5.0


def test_nvt_free_particles_average_temperature():
    """With no forces the thermostat variable oscillates; dxi/dt = (2K - g kT)/Q
    integrates to zero over whole periods, so the time average of 2K/(g kB) is T."""
    rng = np.random.default_rng(3)
    n = 50
    x0 = 500.0 + rng.random((n, 3))
    m = np.full(n, 14.007)
    v0 = rng.normal(size=(n, 3)) * np.sqrt(KAPPA * KB_EV * 600.0 / m[:, None])   # about 600 K

    def ffn(p):
        return 0.0, np.zeros_like(p)

    T, tau = 200.0, 10.0
    o = nose_hoover(ffn, x0, v0, m, np.array([1000.0] * 3), 0.25, 20000, T, tau)
    t_inst = 2.0 * o["ekin"] / (3 * n * KB_EV)
    assert abs(t_inst.mean() / T - 1.0) < 0.03
