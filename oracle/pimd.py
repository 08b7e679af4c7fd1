"""Ring-polymer (path-integral) molecular dynamics (oracle, test infrastructure).

Sec. 6 (Fig. 6): every atom is represented by P replicas (32 in the paper)
coupled harmonically to their neighbours along a closed ring, and the cost
is the energy and forces of every replica.  The paper does not write the
equations or the integrator down.  Reading: the ring-polymer Hamiltonian at
P times the physical temperature,
    H_P = sum_k [ sum_i m_i |v_ik|^2 / 2 + V(q_k) ]
          + sum_i sum_k m_i omega_P^2 |q_ik - q_i,k+1|^2 / 2,
    omega_P = P kB T / hbar,   replica P + 1 = replica 1,
integrated by velocity Verlet with the spring part solved exactly in the
normal modes of the ring (frequencies omega_k = 2 omega_P sin(k pi / P)):
    v += dt/2 kappa F/m;  free ring-polymer evolution for dt;  F <- F(q);
    v += dt/2 kappa F/m,
F the physical force on each replica.  Bead positions are not wrapped into
the box (each bead's neighbour list wraps them), so the springs are plain
differences.  Energies in eV, velocities in A/fs, masses in amu.
"""
import math

import numpy as np

from .md import KAPPA, KB_EV

HBAR_EV_FS = 0.6582119569        # reduced Planck constant, eV fs


def normal_modes(P):
    """Orthogonal C (P x P, C[j, k]: replica j, mode k) and the mode
    frequencies in units of omega_P: mode 0 the centroid; modes
    1 <= k < P/2 cosines, P/2 (P even) the alternating mode, P/2 < k < P
    sines, mode k and P - k sharing 2 sin(k pi / P)."""
    C = np.zeros((P, P))
    w = np.zeros(P)
    j = np.arange(P)
    for k in range(P):
        if k == 0:
            C[:, k] = 1.0 / math.sqrt(P)
        elif 2 * k < P:
            C[:, k] = math.sqrt(2.0 / P) * np.cos(2.0 * math.pi * j * k / P)
        elif 2 * k == P:
            C[:, k] = (-1.0) ** j / math.sqrt(P)
        else:
            C[:, k] = math.sqrt(2.0 / P) * np.sin(2.0 * math.pi * j * k / P)
        kk = k if 2 * k <= P else P - k
        w[k] = 2.0 * math.sin(kk * math.pi / P)
    return C, w


def omega_p(P, temperature):
    """omega_P = P kB T / hbar in 1/fs."""
    return P * KB_EV * temperature / HBAR_EV_FS


def free_ring_step(q, v, dt, wp):
    """Exact evolution of the free ring polymer for dt.  q, v: (P, N, 3)."""
    P = q.shape[0]
    C, w = normal_modes(P)
    qm = np.einsum("jk,jna->kna", C, q)
    vm = np.einsum("jk,jna->kna", C, v)
    for k in range(P):
        om = w[k] * wp
        if om == 0.0:
            qm[k] = qm[k] + dt * vm[k]
        else:
            c, s = math.cos(om * dt), math.sin(om * dt)
            qm[k], vm[k] = c * qm[k] + (s / om) * vm[k], -om * s * qm[k] + c * vm[k]
    return np.einsum("jk,kna->jna", C, qm), np.einsum("jk,kna->jna", C, vm)


def spring_energy(q, masses, wp):
    d = q - np.roll(q, -1, axis=0)
    return 0.5 * wp * wp * float((masses[None, :, None] * d * d).sum()) / KAPPA


def rpmd(force_fn, q, v, masses, dt, n_steps, temperature):
    """n_steps of ring-polymer MD.  q, v: (P, N, 3); force_fn(q_k) -> (V, F)
    for one replica.  Returns dict with final q, v and per-step arrays
    vmean (sum_k V / P), ekin (all replicas) and hp (H_P)."""
    q = np.array(q, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    m = np.asarray(masses, dtype=np.float64)
    P = q.shape[0]
    wp = omega_p(P, temperature)

    def forces(qq):
        out = [force_fn(qq[k]) for k in range(P)]
        return sum(o[0] for o in out), np.stack([np.asarray(o[1], dtype=np.float64) for o in out])

    vsum, F = forces(q)
    rec = {"vmean": [], "ekin": [], "hp": []}
    for _ in range(n_steps):
        v = v + (0.5 * dt) * KAPPA * F / m[None, :, None]
        q, v = free_ring_step(q, v, dt, wp)
        vsum, F = forces(q)
        v = v + (0.5 * dt) * KAPPA * F / m[None, :, None]
        ek = 0.5 * float((m[None, :, None] * v * v).sum()) / KAPPA
        rec["vmean"].append(vsum / P)
        rec["ekin"].append(ek)
        rec["hp"].append(ek + spring_energy(q, m, wp) + vsum)
    for k in rec:
        rec[k] = np.asarray(rec[k])
    rec["q"], rec["v"], rec["forces"] = q, v, F
    return rec
