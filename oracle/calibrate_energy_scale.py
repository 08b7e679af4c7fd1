"""Write tests/golden/energy_scale.json: the per-model energy scale sigma_Z.

Reading (the paper prints no weights): with seeded Gaussian weights the force
scale is arbitrary, so sigma_Z (equal for both species, mu_Z = 0) is chosen
so that the FP64 oracle's RMS force component on the model's first synthetic
frame is 1.0 eV/A, a liquid-NH3-like magnitude that gives an absolute force
tolerance a meaning.  E and F are linear in sigma_Z, so sigma_Z = 1 / RMS(F)
evaluated at sigma_Z = 1.

Run:  python -m oracle.calibrate_energy_scale
Calls only the oracle and the seeded input generators.
"""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
from oracle.model import OracleModel  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "tests", "golden", "energy_scale.json")

# (model name, config, weights seed, molecules in the first frame, frame seed)
CASES = [
    ("tiny", synth.TINY, 42, 16, 0),
    ("tiny_teacher", synth.TINY, 43, 16, 0),
    ("main", synth.MAIN, 42, 1728, 0),
    ("main_teacher", synth.MAIN, 43, 1728, 0),
]


def main():
    torch.set_num_threads(os.cpu_count() or 1)
    out = {"_doc": ("sigma_Z per model so that the FP64 oracle's RMS force component "
                    "on the first frame is 1 eV/A; written by "
                    "oracle/calibrate_energy_scale.py")}
    for name, cfg, wseed, n_mol, fseed in CASES:
        pos, sp, cell = synth.make_ammonia(n_mol, fseed)
        model = OracleModel(synth.make_blob(cfg, wseed, sigma=1.0))
        _, F, _, _ = model.energy_forces(pos, sp, np.diag(cell))
        rms = float(np.sqrt(np.mean(F * F)))
        out[name] = {"weights_seed": wseed, "frame_molecules": n_mol,
                     "frame_seed": fseed, "rms_force_at_sigma_1": rms,
                     "sigma": 1.0 / rms}
        print(name, out[name])
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
