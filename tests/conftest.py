import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build_oracle()
    return oracle


_HCACHE = {}


@pytest.fixture(scope="session")
def hcache(oracle_mod):
    """Session cache of oracle H-matrices keyed by mesh name and build parameters."""
    def get(mesh, leaf=32, eta=2.0, eps=1e-4):
        key = (mesh.name, mesh.n, leaf, eta, eps)
        if key not in _HCACHE:
            _HCACHE[key] = oracle_mod.HMatrix(mesh.centroid, mesh.area, leaf=leaf, eta=eta, eps=eps)
        return _HCACHE[key]
    return get
