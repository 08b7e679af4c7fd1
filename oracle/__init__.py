"""FP64 CPU oracle for the Allegro energy/force hot path (test infrastructure).

This package is the slow, plain reference that the CUDA path is checked
against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it; the library never does, and nothing here imports the library.

What the paper fixes (arXiv 2303.08169):
  * Eq. 1: m_i d^2 r_i/dt^2 = f_i = -dE/dr_i.
  * Sec. 2.1: E is a sum of pairwise embedding energies E_ij inside a finite
    cutoff, built E(3)-equivariantly from tensors up to rank l and tensor
    products of irreducible representations.
  * Eq. 2 / Eq. 3: sharpness and the SAM update.
  * Fig. 1 caption: force outliers are components above 5 sigma.
  * Sec. 3.2: NVE integration; Table 5: Adam (0.9, 0.999), per-atom MSE loss.
The paper does not define the Allegro layers themselves; the concrete
"Allegro-shaped" reading implemented here (Bessel basis, p = 6 envelope, real
spherical harmonics in component normalisation, natural-parity CG paths,
channel-wise tensor products, latent MLPs with 1/sqrt(2) residuals, per-pair
energy MLP) is stated in each function's docstring.

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, library routines (sympy Clebsch-Gordan, scipy Legendre
polynomials), invariances, finite differences and brute force.  The absolute
energy/force values of the whole model have no printed worked example in the
paper; they are pinned only through those properties and the dimer closed
form.
"""
from .blob import read_blob
from .sph import sh_real, real_cg, coupling_paths
from .neighbors import wrap_positions, pairs_bruteforce, pairs_cells, pairs_auto, reverse_index
from .model import OracleModel
from .md import kinetic_energy, outlier_count, velocity_verlet
from .train import loss_and_grad, adam_update, sam_step, flat_params

__all__ = [
    "read_blob", "sh_real", "real_cg", "coupling_paths", "wrap_positions",
    "pairs_bruteforce", "pairs_cells", "pairs_auto", "reverse_index", "OracleModel",
    "kinetic_energy", "outlier_count", "velocity_verlet", "loss_and_grad",
    "adam_update", "sam_step", "flat_params",
]
