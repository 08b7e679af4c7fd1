"""Reader for the "ALW1" weights blob (oracle side, written independently of
the C++ reader).  Layout: magic, 11 u32 header words (the last one the parity
flag: 0 natural-parity paths only, 1 full O(3)), latent and energy widths,
padding to 8 bytes, r_cut, nu, sigma[S], mu[S], a 48-byte-per-entry tensor
directory (name[32], rows, cols, offset) and FP64 row-major tensors.
"""
import struct
import numpy as np


def read_blob(buf):
    """Return (cfg dict, {name: float64 ndarray [rows][cols]}, [names in order])."""
    buf = bytes(buf)
    if buf[:4] != b"ALW1":
        raise ValueError("bad magic")
    (version, S, l_max, n_layers, C, Nb, p, n_lat, n_en, n_t,
     parity) = struct.unpack_from("<11I", buf, 4)
    if version != 1:
        raise ValueError("unsupported version")
    if parity not in (0, 1):
        raise ValueError("parity flag must be 0 or 1")
    off = 48
    latent = struct.unpack_from(f"<{n_lat}I", buf, off)
    off += 4 * n_lat
    energy = struct.unpack_from(f"<{n_en}I", buf, off)
    off += 4 * n_en
    off += (-off) % 8
    r_cut, nu = struct.unpack_from("<2d", buf, off)
    off += 16
    sigma = struct.unpack_from(f"<{S}d", buf, off)
    off += 8 * S
    mu = struct.unpack_from(f"<{S}d", buf, off)
    off += 8 * S
    weights, names = {}, []
    for t in range(n_t):
        raw = buf[off:off + 32]
        name = raw.split(b"\0", 1)[0].decode()
        rows, cols, doff = struct.unpack_from("<IIQ", buf, off + 32)
        off += 48
        arr = np.frombuffer(buf, dtype="<f8", count=rows * cols, offset=doff)
        weights[name] = arr.reshape(rows, cols).astype(np.float64)
        names.append(name)
    cfg = dict(n_species=S, l_max=l_max, n_layers=n_layers, n_channels=C,
               n_bessel=Nb, poly_p=p, latent=tuple(latent), energy=tuple(energy),
               r_cut=r_cut, avg_num_neighbors=nu, sigma=tuple(sigma), mu=tuple(mu), parity=parity)
    return cfg, weights, names
