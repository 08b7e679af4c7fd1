"""Model configurations, seeded Gaussian weights and the weights-blob writer.

Blob format "ALW1" (little-endian), read independently by the oracle and by the
C++ library:

  off  type                 field
    0  char[4]              magic "ALW1"
    4  u32                  version (1)
    8  u32                  n_species S
   12  u32                  l_max
   16  u32                  n_layers L
   20  u32                  n_channels C
   24  u32                  n_bessel Nb
   28  u32                  poly_p (envelope exponent p)
   32  u32                  n_latent  (number of latent hidden widths)
   36  u32                  n_energy  (number of energy-MLP hidden widths)
   40  u32                  n_tensors
   44  u32                  parity: 0 = natural-parity coupling paths only,
                            1 = full O(3) (parity-odd paths and pseudotensor
                            features as well)
   48  u32[n_latent]        latent widths
       u32[n_energy]        energy hidden widths
       (zero padding to an 8-byte boundary)
       f64                  r_cut (Angstrom)
       f64                  avg_num_neighbors (nu)
       f64[S]               sigma_Z (per-species energy scale)
       f64[S]               mu_Z (per-species energy shift)
       n_tensors x 48 B     directory: char name[32] (NUL padded), u32 rows,
                            u32 cols, u64 byte offset of the data
       f64 data             each tensor row-major [rows][cols], 8-byte aligned

Every weight matrix is stored as [fan_out][fan_in]; a layer computes
y = W x / sqrt(fan_in).  Tensor order (= draw order from one seeded
Generator(PCG64(seed)), entries ~ N(0, 1)):

  twobody.0            D0 x (2S + Nb)
  twobody.k            Dk x D(k-1)              k = 1 .. n_latent-1
  embed                C (l_max+1) x D_last
  for layer k = 1 .. L:
    layer{k}.env       C x D_last
    layer{k}.mix{l}    C x (C P_l)              only for k < L, l = 0 .. l_max
    layer{k}.mix{l}p   C x (C Q_kl)             parity 1 only, k < L, every l whose
                                                pseudotensor output has Q_kl > 0 paths
    layer{k}.latent.0  D0 x (D_last + C P_0)
    layer{k}.latent.j  Dj x D(j-1)              j = 1 .. n_latent-1
  energy.0             E0 x D_last
  energy.j             Ej x E(j-1)              j = 1 .. n_energy-1
  energy.out           1 x E_last

P_l counts the coupling paths (l1, l2, l) with l1, l2 <= l_max,
|l1 - l2| <= l <= l1 + l2 and l1 + l2 + l even; it only fixes matrix shapes.
With parity 1 the features of layer k carry irreps (l, s), s = 1 marking the
parity opposite to Y_l's; a path from input (l1, s1) through Y_l2 to output
order l3 lands in s3 = (l1 + s1 + l2 + l3) mod 2, and P_l (for layers k > 1)
and Q_kl count the paths into (l, 0) and (l, 1) from the irreps present
(layer_path_counts); only shapes follow from it here.
"""
import math
import struct
from dataclasses import dataclass, field, replace

import numpy as np

from .ammonia import atoms_per_volume

MAGIC = b"ALW1"
VERSION = 1
NAME_BYTES = 32


def path_counts(l_max):
    """Number of coupling paths ending in each output order l (shape logic only)."""
    counts = [0] * (l_max + 1)
    for l1 in range(l_max + 1):
        for l2 in range(l_max + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, l_max) + 1):
                if (l1 + l2 + l3) % 2 == 0:
                    counts[l3] += 1
    return counts


def layer_path_counts(l_max, parity, n_layers):
    """[{(l3, s3): number of paths}] for layers 1 .. n_layers (shape logic only)."""
    irreps = {(l, 0) for l in range(l_max + 1)}
    out = []
    for _ in range(n_layers):
        cnt = {}
        for (l1, s1) in irreps:
            for l2 in range(l_max + 1):
                for l3 in range(abs(l1 - l2), min(l1 + l2, l_max) + 1):
                    s3 = (l1 + s1 + l2 + l3) % 2
                    if parity == 0 and (s1 or s3):
                        continue
                    cnt[(l3, s3)] = cnt.get((l3, s3), 0) + 1
        out.append(cnt)
        irreps = set(cnt)
    return out


@dataclass(frozen=True)
class ModelConfig:
    r_cut: float
    l_max: int
    n_layers: int
    n_channels: int
    latent: tuple
    energy: tuple
    n_species: int = 2
    n_bessel: int = 8
    poly_p: int = 6
    avg_num_neighbors: float = 0.0
    sigma: tuple = (1.0, 1.0)
    mu: tuple = (0.0, 0.0)
    parity: int = 0

    def with_sigma(self, s):
        return replace(self, sigma=tuple(float(s) for _ in range(self.n_species)))


def _nu(r_cut):
    """Average neighbour count of a uniform liquid at the NH3 atom density."""
    return 4.0 / 3.0 * math.pi * r_cut ** 3 * atoms_per_volume()


# 64-atom model: 1 layer, l_max 1, 8 channels, latent [32, 32], energy [32].
TINY = ModelConfig(r_cut=4.0, l_max=1, n_layers=1, n_channels=8,
                   latent=(32, 32), energy=(32,), avg_num_neighbors=_nu(4.0))
# 6,912 / 110,592 / 1e6-atom model: 2 layers, l_max 2, 16 channels,
# latent [128, 128], energy [32].
MAIN = ModelConfig(r_cut=5.0, l_max=2, n_layers=2, n_channels=16,
                   latent=(128, 128), energy=(32,), avg_num_neighbors=_nu(5.0))


def tensor_shapes(cfg):
    """Ordered list of (name, rows, cols) for the config."""
    S, C, Nb = cfg.n_species, cfg.n_channels, cfg.n_bessel
    D, E = list(cfg.latent), list(cfg.energy)
    counts = layer_path_counts(cfg.l_max, cfg.parity, cfg.n_layers)
    out = [("twobody.0", D[0], 2 * S + Nb)]
    for k in range(1, len(D)):
        out.append((f"twobody.{k}", D[k], D[k - 1]))
    out.append(("embed", C * (cfg.l_max + 1), D[-1]))
    for layer in range(1, cfg.n_layers + 1):
        cnt = counts[layer - 1]
        out.append((f"layer{layer}.env", C, D[-1]))
        if layer < cfg.n_layers:
            for l in range(cfg.l_max + 1):
                out.append((f"layer{layer}.mix{l}", C, C * cnt[(l, 0)]))
            for l in range(cfg.l_max + 1):
                if cnt.get((l, 1), 0) > 0:
                    out.append((f"layer{layer}.mix{l}p", C, C * cnt[(l, 1)]))
        out.append((f"layer{layer}.latent.0", D[0], D[-1] + C * cnt[(0, 0)]))
        for k in range(1, len(D)):
            out.append((f"layer{layer}.latent.{k}", D[k], D[k - 1]))
    out.append(("energy.0", E[0], D[-1]))
    for k in range(1, len(E)):
        out.append((f"energy.{k}", E[k], E[k - 1]))
    out.append(("energy.out", 1, E[-1]))
    return out


def make_weights(cfg, seed):
    """Dict name -> float64 [rows][cols] array of N(0,1) draws, in blob order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return {name: rng.normal(size=(r, c)) for name, r, c in tensor_shapes(cfg)}


def write_blob(cfg, weights):
    shapes = tensor_shapes(cfg)
    S = cfg.n_species
    head = MAGIC + struct.pack(
        "<11I", VERSION, S, cfg.l_max, cfg.n_layers, cfg.n_channels,
        cfg.n_bessel, cfg.poly_p, len(cfg.latent), len(cfg.energy),
        len(shapes), cfg.parity)
    head += struct.pack(f"<{len(cfg.latent)}I", *cfg.latent)
    head += struct.pack(f"<{len(cfg.energy)}I", *cfg.energy)
    head += b"\0" * ((-len(head)) % 8)
    head += struct.pack("<2d", cfg.r_cut, cfg.avg_num_neighbors)
    head += struct.pack(f"<{S}d", *cfg.sigma)
    head += struct.pack(f"<{S}d", *cfg.mu)
    dir_off = len(head)
    data_off = dir_off + 48 * len(shapes)
    directory = b""
    data = b""
    for name, r, c in shapes:
        w = np.ascontiguousarray(weights[name], dtype="<f8")
        assert w.shape == (r, c), (name, w.shape, (r, c))
        nb = name.encode()
        assert len(nb) < NAME_BYTES
        directory += nb + b"\0" * (NAME_BYTES - len(nb))
        directory += struct.pack("<IIQ", r, c, data_off + len(data))
        data += w.tobytes()
    return head + directory + data


def make_blob(cfg, seed, sigma=None):
    """Blob bytes for cfg with weights from seed; sigma overrides sigma_Z."""
    if sigma is not None:
        cfg = cfg.with_sigma(sigma)
    return write_blob(cfg, make_weights(cfg, seed))
