"""NVE velocity Verlet and the force-outlier count (oracle).

Eq. 1 (m_i r_i'' = f_i) integrated microcanonically (Sec. 3.2 runs NVE; the
integrator is not named, the reading is velocity Verlet):
    v += (dt/2) kappa F/m;  r += dt v;  wrap r into [0, L);  F <- F(r);
    v += (dt/2) kappa F/m
with kappa = 1 eV/(A amu) = 9.648533e-3 A/fs^2.
Outliers (Fig. 1 caption: force values "over 5 sigma"): reading: sigma^2 is the
mean of F_ia^2 over all 3N components of the current step (the mean force is
zero), and a component counts when |F_ia| > 5 sigma.
NVT (the runs are equilibrated at 200 K before NVE, Sec. 3.2; the thermostat
is not named): reading: a Nose-Hoover thermostat, g = 3N, Q = g kT tau^2,
integrated with the time-reversible splitting (half thermostat step, velocity
Verlet, half thermostat step); conserved H = E_pot + K + Q xi^2 / 2 + g kT eta.
"""
import numpy as np

from .neighbors import wrap_positions

KAPPA = 9.648533e-3
KB_EV = 8.617333262e-5      # Boltzmann constant, eV/K


def kinetic_energy(vel, masses):
    """sum 1/2 m v^2 in eV (v in A/fs, m in amu)."""
    return 0.5 * float((masses[:, None] * vel * vel).sum()) / KAPPA


def outlier_count(forces, threshold=5.0):
    f = np.asarray(forces, dtype=np.float64).ravel()
    if f.size == 0:
        return 0
    sigma = np.sqrt(np.mean(f * f))
    return int(np.count_nonzero(np.abs(f) > threshold * sigma))


def velocity_verlet(force_fn, pos, vel, masses, lengths, dt, n_steps):
    """Integrate n_steps.  force_fn(pos) -> (E_pot, F).

    Returns dict with final pos/vel and per-step arrays epot, ekin, etot and
    outliers (measured at the end of each step).
    """
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    m = np.asarray(masses, dtype=np.float64)[:, None]
    epot, F = force_fn(pos)
    out = {"epot": [], "ekin": [], "etot": [], "outliers": []}
    for _ in range(n_steps):
        vel = vel + (0.5 * dt) * KAPPA * F / m
        pos = wrap_positions(pos + dt * vel, lengths)
        epot, F = force_fn(pos)
        vel = vel + (0.5 * dt) * KAPPA * F / m
        ek = kinetic_energy(vel, m[:, 0])
        out["epot"].append(epot)
        out["ekin"].append(ek)
        out["etot"].append(epot + ek)
        out["outliers"].append(outlier_count(F))
    out["pos"], out["vel"], out["forces"] = pos, vel, F
    for k in ("epot", "ekin", "etot", "outliers"):
        out[k] = np.asarray(out[k])
    return out


def _thermostat_half(vel, masses, xi, eta, h, gkt, q):
    """One thermostat half step of length h: xi by (h/2) G, velocities scaled
    by exp(-xi h), eta by xi h, xi by (h/2) G with the scaled kinetic energy;
    G = (2K - g kT) / Q."""
    k = kinetic_energy(vel, masses)
    xi = xi + 0.5 * h * (2.0 * k - gkt) / q
    s = np.exp(-xi * h)
    vel = vel * s
    k = k * s * s
    eta = eta + xi * h
    xi = xi + 0.5 * h * (2.0 * k - gkt) / q
    return vel, xi, eta


def nose_hoover(force_fn, pos, vel, masses, lengths, dt, n_steps, temperature, tau, xi=0.0, eta=0.0):
    """NVT: n_steps of (thermostat half step dt/2, velocity Verlet dt,
    thermostat half step dt/2).  force_fn(pos) -> (E_pot, F).  temperature in
    K, tau (thermostat period) in fs.  Returns dict with final pos, vel, xi,
    eta and per-step arrays epot, ekin, etot, hext, outliers."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    mass = np.asarray(masses, dtype=np.float64)
    m = mass[:, None]
    gkt = 3.0 * len(pos) * KB_EV * temperature
    q = gkt * tau * tau
    epot, F = force_fn(pos)
    out = {"epot": [], "ekin": [], "etot": [], "hext": [], "outliers": []}
    for _ in range(n_steps):
        vel, xi, eta = _thermostat_half(vel, mass, xi, eta, 0.5 * dt, gkt, q)
        vel = vel + (0.5 * dt) * KAPPA * F / m
        pos = wrap_positions(pos + dt * vel, lengths)
        epot, F = force_fn(pos)
        vel = vel + (0.5 * dt) * KAPPA * F / m
        vel, xi, eta = _thermostat_half(vel, mass, xi, eta, 0.5 * dt, gkt, q)
        ek = kinetic_energy(vel, mass)
        out["epot"].append(epot)
        out["ekin"].append(ek)
        out["etot"].append(epot + ek)
        out["hext"].append(epot + ek + 0.5 * q * xi * xi + gkt * eta)
        out["outliers"].append(outlier_count(F))
    out["pos"], out["vel"], out["forces"], out["xi"], out["eta"] = pos, vel, F, xi, eta
    for k in ("epot", "ekin", "etot", "hext", "outliers"):
        out[k] = np.asarray(out[k])
    return out
