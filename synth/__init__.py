"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package only draws random numbers and lays them out (liquid-ammonia-shaped
structures, Maxwell-Boltzmann velocities, Gaussian weights and the weights blob
that carries them).  It holds none of the model's arithmetic: no basis
functions, no tensor products, no forces.

Synthetic stand-ins: the paper trains and runs on a liquid-NH3 DFT dataset
(432-atom configurations, Table 5) and on 6,912-atom-per-GPU ammonia systems
(Sec. 3.3); neither is available, so structures are generated at the same
density (0.68 g/cm^3) and molecular geometry, and weights are seeded Gaussians.
"""
from .ammonia import (MASS_AMU, SPECIES_N, SPECIES_H, box_edge, make_ammonia,
                      make_velocities, make_sam_batch, atoms_per_volume)
from .weights import (ModelConfig, TINY, MAIN, path_counts, layer_path_counts, tensor_shapes,
                      make_weights, write_blob, make_blob)

__all__ = [
    "MASS_AMU", "SPECIES_N", "SPECIES_H", "box_edge", "make_ammonia",
    "make_velocities", "make_sam_batch", "atoms_per_volume", "ModelConfig",
    "TINY", "MAIN", "path_counts", "layer_path_counts", "tensor_shapes", "make_weights",
    "write_blob", "make_blob",
]
