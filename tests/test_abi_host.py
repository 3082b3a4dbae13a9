"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every function include/hmat.h declares, the host builder reproduces the
oracle's H-matrix, and blob validation rejects malformed inputs."""
import os
import re

import numpy as np
import pytest

import synth
from blob_util import dense_blob, oracle_blob, read_blob, write_blob

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1911_00093_gb300 as P
    from paper_1911_00093_gb300 import _build
    _build.build()
    P.load()
    return P


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "hmat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmat_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(P):
    names = _declared_functions()
    assert len(names) >= 14
    lib = P.load()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(P.EXPORTS) == names


def test_strerror_covers_every_status(P):
    for st in range(11):
        assert P.hmat_strerror(st) != "unknown status"


@pytest.mark.parametrize("mesh", [synth.icosphere(3), synth.unit_cube(5), synth.two_spheres(2), synth.icosphere(0)],
                         ids=lambda m: m.name)
def test_builder_reproduces_oracle_hmatrix(P, hcache, mesh):
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = hcache(mesh)
    h, perm, cl, bl, data = read_blob(blob)
    idx, _ = H.clusters()
    assert np.array_equal(perm, H.perm)
    assert np.array_equal(cl, idx)
    assert np.array_equal(bl[:, :6], H.blocks[:, :6])
    for b in range(bl.shape[0]):
        d = H.block_data(b)
        flat = d.ravel() if bl[b, 4] == 0 else np.concatenate([d[0].ravel(), d[1].ravel()])
        assert np.array_equal(flat, data[bl[b, 6]:bl[b, 6] + flat.size]), b


def test_builder_arguments(P):
    m = synth.icosphere(1)
    with pytest.raises(P.HmatError):
        P.hmat_build(m.centroid, m.area, leaf=0)
    with pytest.raises(P.HmatError):
        P.hmat_build(m.centroid, m.area, leaf=65)
    with pytest.raises(P.HmatError):
        P.hmat_build(m.centroid, m.area, aca_eps=0.0)
    c = m.centroid.copy(); c[3, 1] = np.nan
    with pytest.raises(P.HmatError):
        P.hmat_build(c, m.area)


def test_stats_of_oracle_blob_and_layout_invariants(P, hcache):
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    st = P.hmat_blob_stats(oracle_blob(H))
    os_ = H.stats()
    assert st["n"] == mesh.n and st["dense_entries"] == os_["dense_entries"] and st["lr_entries"] == os_["lr_entries"]
    assert st["rank_sum"] == os_["rank_sum"] and st["rank_max"] == os_["rank_max"]


def _expect_bad(P, blob, code=2):
    with pytest.raises(P.HmatError) as e:
        P.hmat_blob_stats(blob)
    assert e.value.status == code


def test_validation_rejects_malformed_blobs(P, hcache):
    mesh = synth.icosphere(2)
    H = hcache(mesh)
    good = oracle_blob(H)
    P.hmat_blob_stats(good)
    h, perm, cl, bl, data = read_blob(good)
    blocks = [H.block_data(b) for b in range(bl.shape[0])]
    # bad magic
    b = good.copy(); b[0] = ord("X"); _expect_bad(P, b)
    # truncated
    _expect_bad(P, good[:-64])
    # perm not a permutation
    p2 = perm.copy(); p2[0] = p2[1]
    _expect_bad(P, write_blob(h["n"], p2, cl, bl, blocks))
    # a block dropped: I x J no longer covered (eq. 2)
    keep = np.arange(bl.shape[0]) != 5
    _expect_bad(P, write_blob(h["n"], perm, cl, bl[keep], [blocks[k] for k in np.nonzero(keep)[0]]))
    # a block duplicated: overlap (eq. 1)
    bl2 = np.concatenate([bl, bl[5:6]]); blocks2 = blocks + [blocks[5]]
    _expect_bad(P, write_blob(h["n"], perm, cl, bl2, blocks2))
    # rank larger than min(#I, #J)
    lr = int(np.nonzero(bl[:, 4] == 1)[0][0])
    bl3 = bl.copy(); bl3[lr, 5] = 10 ** 6
    _expect_bad(P, write_blob(h["n"], perm, cl, bl3, blocks))
    # a non-finite value
    blocks4 = list(blocks); d = np.array(blocks4[0], copy=True); d.flat[0] = np.inf; blocks4[0] = d
    _expect_bad(P, write_blob(h["n"], perm, cl, bl, blocks4))
    # leaf larger than the kernels accept
    A = np.eye(70)
    _expect_bad(P, dense_blob(A), code=10)


def test_dense_blob_is_valid(P):
    A = np.array([[2.0, 1.0, -1.0], [-1.0, -1.0, 0.0], [-1.0, 1.0, -1.0]])
    st = P.hmat_blob_stats(dense_blob(A))
    assert st["n"] == 3 and st["dense_entries"] == 9 and st["nleaves"] == 1


def test_product_path_fails_loudly_without_gpu(P):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    mesh = synth.icosphere(1)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    with pytest.raises(P.HmatError):
        P.hmat_upload(blob, "fp64")
