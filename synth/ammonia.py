"""Seeded liquid-ammonia-shaped structures and thermal velocities.

Recipe (stand-in for the paper's liquid-NH3 systems, Sec. 3.2-3.3, Table 5):
  * M molecules in a periodic cubic box whose edge follows from the mass
    density: L = (M * 17.031 g/mol / (rho * N_A * 1e-24))^(1/3) Angstrom with
    rho = 0.68 g/cm^3.
  * Molecule centres on a simple-cubic lattice with n = ceil(M^(1/3)) sites per
    axis (spacing L/n, site centres at (k + 1/2) L/n); the first M sites of a
    seeded permutation are used; each N is jittered by U(-0.1, 0.1) * L/n per
    axis.
  * The three H atoms sit at N + 1.01 A * R h_k, where h_k are the vertices of
    a C3v pyramid whose H-N-H angle is 107 degrees and R is a uniform random
    rotation (normalised Gaussian quaternion).
  * Atom order is N, H, H, H per molecule; species ids N = 0, H = 1.
Positions are returned unwrapped (H atoms may lie outside [0, L)).
All draws use numpy Generator(PCG64(seed)).
"""
import math
import numpy as np

SPECIES_N = 0
SPECIES_H = 1
MASS_AMU = np.array([14.007, 1.008], dtype=np.float64)   # index = species id

NH3_MOLAR_MASS = 17.031          # g/mol
AVOGADRO_E24 = 0.602214          # N_A * 1e-24 (converts g/cm^3 to amu/A^3)
DENSITY = 0.68                   # g/cm^3, liquid ammonia near 200 K
NH_BOND = 1.01                   # Angstrom
HNH_ANGLE_DEG = 107.0
KB_EV = 8.617333e-5              # eV/K
KAPPA = 9.648533e-3              # 1 eV/(A amu) expressed in A/fs^2


def box_edge(n_mol, density=DENSITY):
    """Cubic box edge (Angstrom) holding n_mol NH3 at the given density."""
    return (n_mol * NH3_MOLAR_MASS / (density * AVOGADRO_E24)) ** (1.0 / 3.0)


def atoms_per_volume(density=DENSITY):
    """Atoms per cubic Angstrom of liquid NH3 (4 atoms per molecule)."""
    return 4.0 * density * AVOGADRO_E24 / NH3_MOLAR_MASS


def _lattice_n(n_mol):
    n = 1
    while n ** 3 < n_mol:
        n += 1
    return n


def _rotations(rng, k):
    q = rng.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _pyramid():
    """Unit vectors to the three H atoms of an ideal NH3 (C3v, H-N-H = 107 deg).

    For vertices at polar angle theta around the axis, the H-N-H angle a obeys
    cos a = 1 - 1.5 sin^2 theta.
    """
    cos_a = math.cos(math.radians(HNH_ANGLE_DEG))
    s = math.sqrt((1.0 - cos_a) / 1.5)
    c = math.sqrt(1.0 - s * s)
    phis = [0.0, 2.0 * math.pi / 3.0, 4.0 * math.pi / 3.0]
    return np.array([[s * math.cos(p), s * math.sin(p), c] for p in phis])


def make_ammonia(n_mol, seed, density=DENSITY):
    """Return (positions (4M,3) float64, species (4M,) int32, cell (3,3) float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = box_edge(n_mol, density)
    n = _lattice_n(n_mol)
    spacing = L / n
    sites = rng.permutation(n ** 3)[:n_mol]
    ix, rem = np.divmod(sites, n * n)
    iy, iz = np.divmod(rem, n)
    centres = (np.stack([ix, iy, iz], axis=1) + 0.5) * spacing
    centres = centres + rng.uniform(-0.1, 0.1, size=(n_mol, 3)) * spacing
    R = _rotations(rng, n_mol)
    h = _pyramid()                                     # (3,3)
    hpos = centres[:, None, :] + NH_BOND * np.einsum("mab,kb->mka", R, h)
    pos = np.concatenate([centres[:, None, :], hpos], axis=1).reshape(-1, 3)
    species = np.tile(np.array([SPECIES_N, SPECIES_H, SPECIES_H, SPECIES_H],
                               dtype=np.int32), n_mol)
    cell = np.diag([L, L, L]).astype(np.float64)
    return np.ascontiguousarray(pos), species, cell


def make_velocities(species, temperature, seed, masses=MASS_AMU):
    """Maxwell-Boltzmann velocities in Angstrom/fs.

    Gaussian components with sigma = sqrt(kB T / m) (converted with
    1 eV/amu = KAPPA A^2/fs^2), centre-of-mass velocity removed, then rescaled
    so that sum m v^2 / 2 = (3N - 3)/2 kB T exactly.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    m = masses[species]
    sig = np.sqrt(KB_EV * temperature / m * KAPPA)
    v = rng.normal(size=(len(species), 3)) * sig[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    ke = 0.5 * (m[:, None] * v * v).sum() / KAPPA
    target = 0.5 * (3 * len(species) - 3) * KB_EV * temperature
    if ke > 0:
        v *= math.sqrt(target / ke)
    return np.ascontiguousarray(v)


def make_sam_batch(n_structs=32, size_seed=7, first_seed=1000,
                   min_atoms=64, max_atoms=512, displacement=0.05):
    """A batch of uneven ammonia structures for the SAM training step.

    Sizes are drawn uniform over {min_atoms, min_atoms+4, ..., max_atoms} from
    size_seed; structure b uses seed first_seed + b and is thermally perturbed
    by a Gaussian displacement of displacement * sqrt(1.008 / m) Angstrom per
    component (a 300 K stand-in).  Returns a list of (pos, species, cell).
    """
    rng = np.random.Generator(np.random.PCG64(size_seed))
    choices = np.arange(min_atoms, max_atoms + 1, 4)
    sizes = rng.choice(choices, size=n_structs)
    out = []
    for b, na in enumerate(sizes):
        pos, sp, cell = make_ammonia(int(na) // 4, first_seed + b)
        r2 = np.random.Generator(np.random.PCG64(first_seed + b + 10_000))
        scale = displacement * np.sqrt(MASS_AMU[SPECIES_H] / MASS_AMU[sp])
        pos = pos + r2.normal(size=pos.shape) * scale[:, None]
        out.append((np.ascontiguousarray(pos), sp, cell))
    return out
