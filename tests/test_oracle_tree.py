"""Pins of the oracle's cluster tree and block partition: invariants of the
bisection and the exact-cover property of eq. (1)-(2)."""
import numpy as np
import pytest

import synth


def _check_clusters(H, mesh):
    perm = H.perm
    n = mesh.n
    assert sorted(perm.tolist()) == list(range(n))
    idx, box = H.clusters()
    assert idx[0, 0] == 0 and idx[0, 1] == n
    pts = mesh.centroid[perm]
    for k in range(idx.shape[0]):
        b, e, c0, c1 = idx[k]
        sub = pts[b:e]
        assert np.array_equal(box[k, :3], sub.min(0)) and np.array_equal(box[k, 3:], sub.max(0))
        if c0 < 0:
            assert 1 <= e - b <= H.leaf
            continue
        assert e - b > H.leaf
        lb, le = idx[c0, :2]
        rb, re = idx[c1, :2]
        assert lb == b and le == rb and re == e and le > lb and re > rb
        ext = box[k, 3:] - box[k, :3]
        axis = int(np.argmax(ext))  # first maximum: ties resolved x < y < z
        mid = 0.5 * (box[k, axis] + box[k, 3 + axis])
        left, right = pts[lb:le, axis], pts[rb:re, axis]
        if left.max() <= mid < right.min():
            continue  # midpoint split
        # degenerate midpoint split: median of the (coordinate, index) order
        assert abs((le - lb) - (re - rb)) <= 1
        assert left.max() <= right.min()


def _check_blocks(H, mesh, bitmap):
    n = mesh.n
    blk = H.blocks
    idx, box = H.clusters()
    m = blk[:, 1] - blk[:, 0]
    w = blk[:, 3] - blk[:, 2]
    assert int((m * w).sum()) == n * n           # areas add up to |I x J|
    if bitmap:
        cover = np.zeros((n, n), dtype=np.int32)
        for i_s, i_e, j_s, j_e, *_ in blk:
            cover[i_s:i_e, j_s:j_e] += 1
        assert cover.min() == 1 and cover.max() == 1  # eq. (1) disjoint, eq. (2) covering
    # every block side is a cluster; low-rank blocks are admissible, dense ones are
    # leaf x leaf or admissible blocks that ACA could not compress
    where = {(int(b), int(e)): k for k, (b, e, c0, c1) in enumerate(idx)}
    for i_s, i_e, j_s, j_e, kind, rank, forced in blk:
        t, s = where[(int(i_s), int(i_e))], where[(int(j_s), int(j_e))]
        lo_t, hi_t, lo_s, hi_s = box[t, :3], box[t, 3:], box[s, :3], box[s, 3:]
        gap = np.maximum(0, np.maximum(lo_s - hi_t, lo_t - hi_s))
        dist = np.sqrt((gap ** 2).sum())
        diam = min(np.linalg.norm(hi_t - lo_t), np.linalg.norm(hi_s - lo_s))
        adm = dist > 0 and diam <= H.eta * dist
        if kind == 1:
            assert adm and 0 < rank < min(i_e - i_s, j_e - j_s)
            assert rank * ((i_e - i_s) + (j_e - j_s)) < (i_e - i_s) * (j_e - j_s)
        elif forced:
            assert adm
        else:
            assert not adm and idx[t, 2] < 0 and idx[s, 2] < 0


@pytest.mark.parametrize("level,bitmap", [(1, True), (2, True), (3, True), (4, False)])
def test_icosphere_tree_and_partition(hcache, level, bitmap):
    mesh = synth.icosphere(level)
    H = hcache(mesh)
    _check_clusters(H, mesh)
    _check_blocks(H, mesh, bitmap)


def test_cube_tree_with_ties(hcache):
    # the cube grid puts many collocation points on one plane: exercises ties and
    # degenerate splits
    mesh = synth.unit_cube(6)
    H = hcache(mesh)
    _check_clusters(H, mesh)
    _check_blocks(H, mesh, True)


def test_admissibility_helper(oracle_mod):
    a = ([0, 0, 0], [1, 1, 1])
    far = ([4, 0, 0], [5, 1, 1])
    near = ([1.5, 0, 0], [2.5, 1, 1])
    touch = ([1, 0, 0], [2, 1, 1])
    assert oracle_mod.admissible(a, far, 2.0)       # diam sqrt3 <= 2 * 3
    assert not oracle_mod.admissible(a, near, 2.0)  # sqrt3 > 2 * 0.5
    assert not oracle_mod.admissible(a, touch, 2.0)  # touching boxes are never admissible
    pt = ([0, 0, 0], [0, 0, 0])
    assert not oracle_mod.admissible(pt, pt, 2.0)


def test_eta_zero_gives_all_dense(oracle_mod):
    mesh = synth.icosphere(2)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area, eta=0.0)
    assert (H.blocks[:, 4] == 0).all()
