"""Host-only checks of the C ABI: the library builds, loads, exports every
function declared in include/allegro.h, and rejects malformed input before
touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
import paper_2303_08169_gb300 as al
from paper_2303_08169_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    return al.lib()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(allegro_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(built):
    declared = _declared()
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(built, name), name
    assert set(declared) == set(al.EXPORTED) | (set(declared) - set(al.EXPORTED))
    assert set(al.EXPORTED) <= set(declared)


def test_version(built):
    assert al.allegro_version().startswith("allegro-gb300")


def test_bad_blob_and_mismatch_rejected_on_host(built):
    mass = np.array([14.007, 1.008])
    with pytest.raises(al.AllegroError) as e:
        al.allegro_create(b"NOPE" + b"\0" * 100, mass, 4.0, 1, 1)
    assert e.value.code == 11
    blob = synth.make_blob(synth.TINY, 1)
    with pytest.raises(al.AllegroError) as e:
        al.allegro_create(blob, mass, 4.5, 1, 1)          # r_cut disagrees
    assert e.value.code == 2
    with pytest.raises(al.AllegroError) as e:
        al.allegro_create(blob[:200], mass, 4.0, 1, 1)    # truncated
    assert e.value.code == 11
    odd = synth.ModelConfig(r_cut=4.0, l_max=1, n_layers=1, n_channels=4, latent=(8, 8), energy=(8,))
    with pytest.raises(al.AllegroError) as e:
        al.allegro_create(synth.make_blob(odd, 1), mass, 4.0, 1, 1)
    assert e.value.code == 10


def test_full_o3_blobs_on_host(built):
    """The parity flag: a three-layer full-O(3) blob whose pseudotensor
    mixing matrix does not have one column per path of the layer's input
    irreps (layer 2, block (1, odd): 5 paths, (0, odd) is no input there), and
    an out-of-range flag, are malformed blobs (E_BLOB), both before any GPU
    work."""
    import dataclasses
    from synth.weights import NAME_BYTES
    mass = np.array([14.007, 1.008])
    cfg3 = dataclasses.replace(synth.MAIN, n_layers=3, parity=1)
    blob = bytearray(synth.make_blob(cfg3, 1))
    off = blob.index(b"layer2.mix1p\0") + NAME_BYTES + 4          # directory entry: rows, cols, offset
    assert int.from_bytes(blob[off:off + 4], "little") == cfg3.n_channels * 5
    blob[off:off + 4] = (cfg3.n_channels * 4).to_bytes(4, "little")
    with pytest.raises(al.AllegroError) as e:
        al.allegro_create(bytes(blob), mass, cfg3.r_cut, cfg3.l_max, 3)
    assert e.value.code == 11
    # well-formed full-O(3) blobs of every compiled shape pass the blob and
    # shape checks (without a GPU, creation then stops at the first device
    # allocation)
    for base, l_max, n_layers in [(synth.TINY, 1, 3), (synth.TINY, 1, 4), (synth.MAIN, 1, 3), (synth.MAIN, 2, 3),
                                  (synth.MAIN, 2, 4), (synth.MAIN, 0, 3)]:
        cfg = dataclasses.replace(base, l_max=l_max, n_layers=n_layers, parity=1)
        try:
            al.allegro_destroy(al.allegro_create(synth.make_blob(cfg, 2), mass, cfg.r_cut, l_max, n_layers))
        except al.AllegroError as err:
            assert err.code in (6, 9), (base, l_max, n_layers, err)        # E_OOM, E_CUDA
    blob = bytearray(synth.make_blob(synth.MAIN, 1))
    blob[44:48] = (2).to_bytes(4, "little")
    with pytest.raises(al.AllegroError) as e:
        al.allegro_create(bytes(blob), mass, synth.MAIN.r_cut, 2, 2)
    assert e.value.code == 11


def test_binding_checks_element_types_and_counts(built):
    """The C entry points take typed pointers without sizes: the binding
    converts host input arrays to the declared element type and rejects a
    device tensor (here a CPU tensor, checked before any library call) or an
    output of the wrong type or size, instead of letting the library
    reinterpret it (an int64 species array read as int32 makes every other
    atom species 0)."""
    import torch
    pos = np.zeros((4, 3))
    with pytest.raises(TypeError):
        al.allegro_energy_forces(None, torch.zeros((4, 3), dtype=torch.float64),
                                 torch.zeros(4, dtype=torch.int64), np.eye(3) * 20.0)
    with pytest.raises(TypeError):
        al.allegro_energy_forces(None, pos, np.zeros(4, np.int32), np.eye(3) * 20.0,
                                 torch.zeros((4, 3), dtype=torch.float64))
    with pytest.raises(ValueError):
        al.allegro_energy_forces(None, pos, np.zeros(4, np.int32), np.eye(3) * 20.0,
                                 np.zeros((3, 3), np.float32))
    with pytest.raises(ValueError):
        al.allegro_md_init(None, pos, np.zeros((4, 3)), torch.zeros(5, dtype=torch.int32), np.eye(3) * 20.0)
    # host inputs of another type are converted; the NULL context is then
    # rejected by the library itself
    with pytest.raises(al.AllegroError) as e:
        al.allegro_energy_forces(None, pos.astype(np.float32), np.zeros(4, np.int64), np.eye(3) * 20.0)
    assert e.value.code == 1


def test_null_arguments(built):
    out = ctypes.c_void_p()
    rc = built.allegro_create(None, 0, None, 2, 4.0, 1, 1, ctypes.byref(out))
    assert rc == 1
    assert built.allegro_set_stream(None, None) == 1
    assert built.allegro_md_step_nve(None, 1.0, 1, None, None) == 1
    assert built.allegro_pimd_step(None, 1.0, 1, None) == 1
    assert built.allegro_pimd_get_state(None, None, None) == 1
    assert built.allegro_pimd_init(None, 4, 10, None, None, None, None, 200.0) == 1


def test_torch_glue_is_autograd_functions():
    """The torch glue is two autograd Functions over the library calls (no
    compute of its own)."""
    import torch
    from paper_2303_08169_gb300 import torch_ops
    assert issubclass(torch_ops.EnergyFunction, torch.autograd.Function)
    assert issubclass(torch_ops.BatchLossFunction, torch.autograd.Function)
    assert callable(torch_ops.energy) and callable(torch_ops.batch_loss)
