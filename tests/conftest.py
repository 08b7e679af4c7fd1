import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def energy_scale(name):
    with open(os.path.join(GOLDEN, "energy_scale.json")) as f:
        return json.load(f)[name]["sigma"]


@pytest.fixture(scope="session")
def tiny_blob():
    import synth
    return synth.make_blob(synth.TINY, 42, sigma=energy_scale("tiny"))


@pytest.fixture(scope="session")
def main_blob():
    import synth
    return synth.make_blob(synth.MAIN, 42, sigma=energy_scale("main"))


@pytest.fixture(scope="session")
def tiny_model(tiny_blob):
    from oracle import OracleModel
    return OracleModel(tiny_blob)
