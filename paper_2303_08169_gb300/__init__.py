"""Python binding of the GB300 Allegro library (include/allegro.h).

Argument marshalling only: every function forwards numpy arrays or torch
tensors (host or CUDA) as raw pointers to the C ABI of the same name.  All
computation runs in the library's CUDA kernels; there is no Python or CPU
fallback, and importing the functions fails loudly when the library has not
been built (see build_lib.build()).
"""
import ctypes
import os

import numpy as np

from .build_lib import LIB, build

ALLEGRO_FP32 = 0
ALLEGRO_BF16 = 1
ALLEGRO_FP16 = 2
ALLEGRO_FP16_SPLIT = 3

_STATUS = {
    0: "OK", 1: "E_INVALID_ARG", 2: "E_MISMATCH", 3: "E_CUTOFF_TOO_LARGE",
    4: "E_NONORTHO_CELL", 5: "E_PAIR_OVERFLOW", 6: "E_OOM", 7: "E_NONFINITE",
    8: "E_TIMEOUT", 9: "E_CUDA", 10: "E_UNSUPPORTED", 11: "E_BLOB",
}

EXPORTED = [
    "allegro_version", "allegro_create", "allegro_destroy", "allegro_set_stream",
    "allegro_last_error", "allegro_build_neighbors", "allegro_get_neighbors",
    "allegro_energy_forces", "allegro_outlier_count", "allegro_md_init",
    "allegro_set_md_precision", "allegro_md_step_nve", "allegro_md_get_state",
    "allegro_query", "allegro_phase_times", "allegro_selftest_mma",
    "allegro_selftest_mma_mode", "allegro_outlier_count_noalloc",
    "allegro_loss_grad", "allegro_sam_train_step", "allegro_get_weights", "allegro_set_weights",
    "allegro_loss_scan", "allegro_md_step_nvt", "allegro_md_get_thermostat",
    "allegro_pimd_init", "allegro_pimd_step", "allegro_pimd_get_state",
    "allegro_debug_inject_wait_timeout", "allegro_selftest_silu", "allegro_set_skin",
]

ALLEGRO_Q_N_PAIRS = 0
ALLEGRO_Q_CAPACITY = 1
ALLEGRO_Q_STEP_KERNELS = 2
ALLEGRO_Q_N_ATOMS = 3
ALLEGRO_Q_N_PARAMS = 4
ALLEGRO_Q_RP_STEP_KERNELS = 5
ALLEGRO_Q_BATCH_PAIRS = 6
ALLEGRO_Q_REBUILDS = 7
ALLEGRO_Q_FP32_LAUNCH = 8
ALLEGRO_Q_TANGENT_LAUNCH = 9


class _Batch(ctypes.Structure):
    _fields_ = [("n_structs", ctypes.c_int32), ("atom_offset", ctypes.c_void_p),
                ("positions", ctypes.c_void_p), ("species", ctypes.c_void_p),
                ("cells", ctypes.c_void_p), ("e_target", ctypes.c_void_p),
                ("f_target", ctypes.c_void_p)]
PHASES = ["neighbors", "pass_a", "pass_b", "pass_c", "pass_b_adjoint", "pass_a_adjoint", "forces",
          "pass_b1", "pass_b2"]


class AllegroError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

_vp, _i32, _i64, _f64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is missing: build it with paper_2303_08169_gb300.build()")
    L = ctypes.CDLL(LIB)
    sig = {
        "allegro_version": ([], ctypes.c_char_p),
        "allegro_create": ([_vp, _sz, _vp, _i32, _f64, _i32, _i32, ctypes.POINTER(_vp)], ctypes.c_int),
        "allegro_destroy": ([_vp], None),
        "allegro_set_stream": ([_vp, _vp], ctypes.c_int),
        "allegro_last_error": ([_vp], ctypes.c_char_p),
        "allegro_build_neighbors": ([_vp, _i64, _vp, _vp, ctypes.POINTER(_i64)], ctypes.c_int),
        "allegro_get_neighbors": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "allegro_energy_forces": ([_vp, _i64, _vp, _vp, _vp, ctypes.POINTER(_f64), _vp, _vp, _i32], ctypes.c_int),
        "allegro_outlier_count": ([_vp, _i64, _vp, _f64, ctypes.POINTER(_i64)], ctypes.c_int),
        "allegro_md_init": ([_vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
        "allegro_set_md_precision": ([_vp, _i32], ctypes.c_int),
        "allegro_md_step_nve": ([_vp, _f64, _i32, _vp, _vp], ctypes.c_int),
        "allegro_md_step_nvt": ([_vp, _f64, _i32, _f64, _f64, _vp, _vp], ctypes.c_int),
        "allegro_md_get_thermostat": ([_vp, _vp], ctypes.c_int),
        "allegro_pimd_init": ([_vp, _i32, _i64, _vp, _vp, _vp, _vp, _f64], ctypes.c_int),
        "allegro_pimd_step": ([_vp, _f64, _i32, _vp], ctypes.c_int),
        "allegro_pimd_get_state": ([_vp, _vp, _vp], ctypes.c_int),
        "allegro_md_get_state": ([_vp, _vp, _vp, _vp, ctypes.POINTER(_i64)], ctypes.c_int),
        "allegro_query": ([_vp, _i32, ctypes.POINTER(_i64)], ctypes.c_int),
        "allegro_phase_times": ([_vp, _i32, _vp, _i32], ctypes.c_int),
        "allegro_selftest_mma": ([_i32, _i32, _vp, _vp, _vp], ctypes.c_int),
        "allegro_selftest_mma_mode": ([_i32, _i32, _vp, _vp, _vp, _i32], ctypes.c_int),
        "allegro_outlier_count_noalloc": ([_i64, _vp, _f64, _vp, _vp], ctypes.c_int),
        "allegro_loss_grad": ([_vp, _vp, _f64, _f64, ctypes.POINTER(_f64), _vp], ctypes.c_int),
        "allegro_sam_train_step": ([_vp, _vp, _f64, _f64, _f64, _f64, ctypes.POINTER(_f64)], ctypes.c_int),
        "allegro_loss_scan": ([_vp, _vp, _vp, _i64, _vp, _i32, _f64, _f64, _vp], ctypes.c_int),
        "allegro_get_weights": ([_vp, _vp, _i64], ctypes.c_int),
        "allegro_set_weights": ([_vp, _vp, _i64], ctypes.c_int),
        "allegro_debug_inject_wait_timeout": ([_i32], ctypes.c_int),
        "allegro_selftest_silu": ([_i64, _vp, _vp], ctypes.c_int),
        "allegro_set_skin": ([_vp, _f64], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(x, dtype=None, count=None, name="array"):
    """Raw address of a numpy array / torch tensor (None -> NULL).  The
    library takes typed pointers without sizes, so the element type (dtype:
    'float64', 'float32', 'int32', 'int64', 'int8') and, where given, the
    number of elements are checked here: a mismatch raises instead of being
    reinterpreted by the library."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: arrays must be C-contiguous")
        kind, size, addr = str(x.dtype), int(x.size), x.ctypes.data
    elif hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError(f"{name}: tensors must be contiguous")
        kind, size, addr = str(x.dtype).replace("torch.", ""), int(x.numel()), x.data_ptr()
    else:
        raise TypeError(f"{name}: unsupported array type {type(x)}")
    if dtype is not None and kind != dtype:
        raise TypeError(f"{name}: element type {kind}, expected {dtype}")
    if count is not None and size != count:
        raise ValueError(f"{name}: {size} elements, expected {count}")
    return addr


def _host(x, dtype):
    return None if x is None else np.ascontiguousarray(x, dtype=dtype)


def _in(x, dtype):
    """An input array: a host numpy array is converted to dtype (the library
    copies host inputs anyway); a device tensor is passed as it is and its
    element type is checked by _ptr."""
    return np.ascontiguousarray(x, dtype=dtype) if isinstance(x, np.ndarray) else x


def _check(ctx, rc):
    if rc != 0:
        msg = lib().allegro_last_error(ctx)
        raise AllegroError(rc, msg.decode() if msg else "")


def allegro_version():
    return lib().allegro_version().decode()


def allegro_create(blob, species_mass, r_cut, l_max, n_layers):
    blob = bytes(blob)
    mass = _host(species_mass, np.float64)
    out = _vp()
    buf = ctypes.create_string_buffer(blob, len(blob))
    rc = lib().allegro_create(ctypes.cast(buf, _vp), len(blob), _ptr(mass), len(mass), float(r_cut),
                              int(l_max), int(n_layers), ctypes.byref(out))
    _check(None, rc)
    return out


def allegro_destroy(ctx):
    lib().allegro_destroy(ctx)


def allegro_set_stream(ctx, stream):
    """stream: torch.cuda.Stream, an integer cudaStream_t, or None."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(ctx, lib().allegro_set_stream(ctx, handle))


def allegro_build_neighbors(ctx, positions, cell):
    positions = _in(positions, np.float64)
    n = int(positions.shape[0])
    cell = _host(cell, np.float64)
    np_ = _i64()
    _check(ctx, lib().allegro_build_neighbors(ctx, n, _ptr(positions, "float64", 3 * n, "positions"), _ptr(cell),
                                              ctypes.byref(np_)))
    return np_.value


def allegro_get_neighbors(ctx, row_ptr=None, col=None, img=None, rev=None):
    _check(ctx, lib().allegro_get_neighbors(ctx, _ptr(row_ptr, "int32", name="row_ptr"), _ptr(col, "int32", name="col"),
                                            _ptr(img, "int8", name="img"), _ptr(rev, "int32", name="rev")))


def allegro_energy_forces(ctx, positions, species, cell, forces_out=None, atom_energy=None,
                          precision=ALLEGRO_FP32):
    positions, species = _in(positions, np.float64), _in(species, np.int32)
    n = int(positions.shape[0])
    cell = _host(cell, np.float64)
    e = _f64()
    _check(ctx, lib().allegro_energy_forces(ctx, n, _ptr(positions, "float64", 3 * n, "positions"),
                                            _ptr(species, "int32", n, "species"), _ptr(cell), ctypes.byref(e),
                                            _ptr(forces_out, "float32", 3 * n, "forces_out"),
                                            _ptr(atom_energy, "float64", n, "atom_energy"), int(precision)))
    return e.value


def allegro_outlier_count(ctx, forces, threshold=5.0):
    forces = _in(forces, np.float32)
    c = _i64()
    n = int(forces.shape[0])
    _check(ctx, lib().allegro_outlier_count(ctx, n, _ptr(forces, "float32", 3 * n, "forces"), float(threshold),
                                            ctypes.byref(c)))
    return c.value


def allegro_md_init(ctx, positions, velocities, species, cell):
    positions, velocities, species = _in(positions, np.float64), _in(velocities, np.float64), _in(species, np.int32)
    cell = _host(cell, np.float64)
    n = int(positions.shape[0])
    _check(ctx, lib().allegro_md_init(ctx, n, _ptr(positions, "float64", 3 * n, "positions"),
                                      _ptr(velocities, "float64", 3 * n, "velocities"),
                                      _ptr(species, "int32", n, "species"), _ptr(cell)))


def allegro_outlier_count_noalloc(forces, threshold, count_out, stream=None):
    """Outlier count into the device int64 count_out, with no device
    allocation (see include/allegro.h); enqueued on stream, not synchronised."""
    handle = getattr(stream, "cuda_stream", stream)
    n = int(forces.shape[0])
    _check(None, lib().allegro_outlier_count_noalloc(n, _ptr(forces, "float32", 3 * n, "forces"), float(threshold),
                                                     _ptr(count_out, "int64", 1, "count_out"), handle))


def make_batch(structs):
    """Host arrays of an allegro_batch from a list of dicts with keys pos,
    species, cell (3x3), e_target, f_target.  Returns (batch, keepalive)."""
    off = np.zeros(len(structs) + 1, dtype=np.int64)
    for k, s in enumerate(structs):
        off[k + 1] = off[k] + len(s["species"])
    pos = np.ascontiguousarray(np.concatenate([s["pos"] for s in structs]), dtype=np.float64)
    sp = np.ascontiguousarray(np.concatenate([s["species"] for s in structs]), dtype=np.int32)
    cells = np.ascontiguousarray(np.stack([np.asarray(s["cell"], dtype=np.float64).reshape(9) for s in structs]))
    et = np.ascontiguousarray([float(s["e_target"]) for s in structs], dtype=np.float64)
    ft = np.ascontiguousarray(np.concatenate([s["f_target"] for s in structs]), dtype=np.float32)
    keep = (off, pos, sp, cells, et, ft)
    b = _Batch(len(structs), off.ctypes.data, pos.ctypes.data, sp.ctypes.data, cells.ctypes.data,
               et.ctypes.data, ft.ctypes.data)
    return b, keep


def allegro_loss_grad(ctx, batch, w_energy=1.0, w_force=100.0, grad_out=None):
    loss = _f64()
    _check(ctx, lib().allegro_loss_grad(ctx, ctypes.byref(batch), float(w_energy), float(w_force),
                                        ctypes.byref(loss), _ptr(grad_out, "float32", name="grad_out")))
    return loss.value


def allegro_sam_train_step(ctx, batch, rho, lr, w_energy=1.0, w_force=100.0):
    loss = _f64()
    _check(ctx, lib().allegro_sam_train_step(ctx, ctypes.byref(batch), float(rho), float(lr), float(w_energy),
                                             float(w_force), ctypes.byref(loss)))
    return loss.value


def allegro_loss_scan(ctx, batch, dirs, scales, w_energy=1.0, w_force=100.0):
    """Loss at w + scales[k] * dirs[k] (dirs: device tensor, one row per
    point, or one row shared by every point); returns a numpy array."""
    scales = np.ascontiguousarray(np.asarray(scales, dtype=np.float64).reshape(-1))
    stride = 0 if dirs.dim() == 1 or dirs.shape[0] == 1 else int(dirs.shape[1])
    if stride and dirs.shape[0] != scales.shape[0]:
        raise ValueError("one direction per scale, or one direction for all")
    out = np.zeros(scales.shape[0], dtype=np.float64)
    d = dirs.contiguous()                             # kept alive across the call
    _check(ctx, lib().allegro_loss_scan(ctx, ctypes.byref(batch), _ptr(d, "float32", name="dirs"), stride, _ptr(scales),
                                        int(scales.shape[0]), float(w_energy), float(w_force), _ptr(out)))
    return out


def allegro_get_weights(ctx, out):
    _check(ctx, lib().allegro_get_weights(ctx, _ptr(out, "float32", name="out"), int(out.shape[0])))


def allegro_set_weights(ctx, w):
    w = _in(w, np.float32)
    _check(ctx, lib().allegro_set_weights(ctx, _ptr(w, "float32", name="weights"), int(w.shape[0])))


def allegro_set_md_precision(ctx, precision):
    _check(ctx, lib().allegro_set_md_precision(ctx, int(precision)))


def allegro_md_step_nve(ctx, dt_fs, n_steps, outlier_counts=None, energies=None):
    n = int(n_steps)
    _check(ctx, lib().allegro_md_step_nve(ctx, float(dt_fs), n, _ptr(outlier_counts, "int64", n, "outlier_counts"),
                                          _ptr(energies, "float64", 3 * n, "energies")))


def allegro_md_step_nvt(ctx, dt_fs, n_steps, temperature_K, tau_fs, outlier_counts=None, energies=None):
    """energies: (n_steps, 4) FP64 (E_pot, E_kin, E_tot, H) or None."""
    n = int(n_steps)
    _check(ctx, lib().allegro_md_step_nvt(ctx, float(dt_fs), n, float(temperature_K), float(tau_fs),
                                          _ptr(outlier_counts, "int64", n, "outlier_counts"),
                                          _ptr(energies, "float64", 4 * n, "energies")))


def allegro_md_get_thermostat(ctx):
    """(xi, eta) of the Nose-Hoover thermostat."""
    out = np.zeros(2, dtype=np.float64)
    _check(ctx, lib().allegro_md_get_thermostat(ctx, _ptr(out)))
    return float(out[0]), float(out[1])


def allegro_pimd_init(ctx, positions, velocities, species, cell, temperature_K):
    """positions, velocities: (P, N, 3) FP64 (host or device); species (N,)."""
    positions, velocities, species = _in(positions, np.float64), _in(velocities, np.float64), _in(species, np.int32)
    cell = _host(cell, np.float64)
    P, n = int(positions.shape[0]), int(positions.shape[1])
    _check(ctx, lib().allegro_pimd_init(ctx, P, n, _ptr(positions, "float64", 3 * P * n, "positions"),
                                        _ptr(velocities, "float64", 3 * P * n, "velocities"),
                                        _ptr(species, "int32", n, "species"), _ptr(cell), float(temperature_K)))


def allegro_pimd_step(ctx, dt_fs, n_steps, energies=None):
    """energies: (n_steps, 3) FP64 (mean replica energy, kinetic, H_P) or None."""
    _check(ctx, lib().allegro_pimd_step(ctx, float(dt_fs), int(n_steps), _ptr(energies, "float64", 3 * int(n_steps), "energies")))


def allegro_pimd_get_state(ctx, positions=None, velocities=None):
    _check(ctx, lib().allegro_pimd_get_state(ctx, _ptr(positions, "float64", name="positions"),
                                             _ptr(velocities, "float64", name="velocities")))


def allegro_md_get_state(ctx, positions=None, velocities=None, forces=None):
    s = _i64()
    _check(ctx, lib().allegro_md_get_state(ctx, _ptr(positions, "float64", name="positions"),
                                           _ptr(velocities, "float64", name="velocities"),
                                           _ptr(forces, "float32", name="forces"), ctypes.byref(s)))
    return s.value


def allegro_query(ctx, what):
    v = _i64()
    _check(ctx, lib().allegro_query(ctx, int(what), ctypes.byref(v)))
    return v.value


def allegro_phase_times(ctx, n_reps=10):
    """Mean ms per phase (keys of PHASES) of one energy+forces evaluation."""
    out = np.zeros(len(PHASES))
    _check(ctx, lib().allegro_phase_times(ctx, int(n_reps), _ptr(out), len(PHASES)))
    return dict(zip(PHASES, out.tolist()))


def allegro_selftest_mma(a, b, d):
    """d (128 x n) = bf16(a) (128 x k) @ bf16(b)^T (n x k), all CUDA float32 tensors."""
    _check(None, lib().allegro_selftest_mma(int(b.shape[0]), int(b.shape[1]), _ptr(a), _ptr(b), _ptr(d)))


def allegro_selftest_mma_mode(a, b, d, mode):
    """mode 0: d = a @ b^T (b: n x k); modes 1, 2: d = a @ b (b: k x n, MN-major read)."""
    n, k = (b.shape[0], b.shape[1]) if mode == 0 else (b.shape[1], b.shape[0])
    _check(None, lib().allegro_selftest_mma_mode(int(n), int(k), _ptr(a), _ptr(b), _ptr(d), int(mode)))


__all__ = ["ALLEGRO_FP32", "ALLEGRO_BF16", "ALLEGRO_FP16", "ALLEGRO_FP16_SPLIT", "AllegroError", "EXPORTED", "build", "lib"] + EXPORTED


def allegro_debug_inject_wait_timeout(enable):
    """Failure injection for tests: the tensor-core passes skip their weight
    copies and their bounded waits run out (ALLEGRO_E_TIMEOUT)."""
    _check(None, lib().allegro_debug_inject_wait_timeout(int(bool(enable))))


def allegro_selftest_silu(x, y):
    """y[2i], y[2i+1] = SiLU(x[i]), SiLU'(x[i]) as the tensor-core passes
    compute them (device tensors: x n FP32, y 2n FP32)."""
    _check(None, lib().allegro_selftest_silu(int(x.numel()), _ptr(x), _ptr(y)))


def allegro_set_skin(ctx, skin_A):
    """Verlet-skin reuse of the MD neighbour list (0 = rebuild every step);
    takes effect at the next allegro_md_init."""
    _check(ctx, lib().allegro_set_skin(ctx, float(skin_A)))
