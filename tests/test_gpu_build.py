"""H-matrix construction on the device (hmat_build_device): the ACA of every
admissible block and the dense entries computed by the GPU must give the host
builder's blob byte for byte (the same operations in the same order), and so
the oracle's own H-matrix, which the host builder reproduces exactly."""
import numpy as np
import pytest

import synth
from blob_util import read_blob
from gpu_util import lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh", [synth.icosphere(0), synth.icosphere(3), synth.unit_cube(8), synth.two_spheres(3),
                                  synth.icosphere(4)], ids=lambda m: m.name)
def test_device_build_is_the_host_blob(hcache, mesh):
    need_gpu()
    P = lib()
    host = P.hmat_build(mesh.centroid, mesh.area)
    info = {}
    dev = P.hmat_build_device(mesh.centroid, mesh.area, info=info)
    assert dev.shape == host.shape and np.array_equal(dev, host)
    assert info["host_blocks"] == 0
    # and the oracle's H-matrix (blocks, ranks and every factor value)
    H = hcache(mesh)
    _, perm, _, bl, data = read_blob(dev)
    assert np.array_equal(perm, H.perm) and np.array_equal(bl[:, :6], H.blocks[:, :6])
    for b in np.random.default_rng(mesh.n).choice(bl.shape[0], min(64, bl.shape[0]), replace=False):
        d = H.block_data(b)
        flat = d.ravel() if bl[b, 4] == 0 else np.concatenate([d[0].ravel(), d[1].ravel()])
        assert np.array_equal(flat, data[bl[b, 6]:bl[b, 6] + flat.size]), b


@pytest.mark.parametrize("leaf,eta,eps", [(16, 1.0, 1e-6), (64, 3.0, 1e-2), (32, 2.0, 1e-12)])
def test_device_build_other_parameters(leaf, eta, eps):
    """Other leaf sizes, admissibility and ACA accuracies (1e-12 drives ranks
    towards the 64 the device workspace holds; blocks beyond it are finished by
    the host builder's code, and the blob is still the host's)."""
    need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    host = P.hmat_build(mesh.centroid, mesh.area, leaf=leaf, eta=eta, aca_eps=eps)
    info = {}
    dev = P.hmat_build_device(mesh.centroid, mesh.area, leaf=leaf, eta=eta, aca_eps=eps, info=info)
    assert np.array_equal(dev, host), info
    assert info["aca_blocks"] > 0


def test_device_build_arguments():
    need_gpu()
    P = lib()
    m = synth.icosphere(1)
    for kw in ({"leaf": 0}, {"leaf": 65}, {"aca_eps": 0.0}, {"eta": -1.0}):
        with pytest.raises(P.HmatError) as e:
            P.hmat_build_device(m.centroid, m.area, **kw)
        assert e.value.status == 1
    c = m.centroid.copy()
    c[3, 1] = np.nan
    with pytest.raises(P.HmatError):
        P.hmat_build_device(c, m.area)


def test_device_build_full_size():
    """Icosphere level 6 (N = 81,920): the device blob is the host blob."""
    need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    info = {}
    dev = P.hmat_build_device(mesh.centroid, mesh.area, info=info)
    host = P.hmat_build(mesh.centroid, mesh.area)
    assert np.array_equal(dev, host), info
    assert info["host_blocks"] == 0 and info["aca_blocks"] > 10000
