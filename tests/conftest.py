import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def geom_full():
    from synth.geometry import make_geometry
    return make_geometry(barrel_only=False)


@pytest.fixture(scope="session")
def geom_barrel():
    from synth.geometry import make_geometry
    return make_geometry(barrel_only=True)


@pytest.fixture(scope="session")
def maps_full(geom_full):
    from synth.maps import load_maps
    return load_maps(geom_full)


@pytest.fixture(scope="session")
def maps_barrel(geom_barrel):
    from synth.maps import load_maps
    return load_maps(geom_barrel)


@pytest.fixture(scope="session")
def cuts():
    from synth.config import DEFAULT_CUTS
    return dict(DEFAULT_CUTS)
