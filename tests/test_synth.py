"""Seeded input generators: geometry facts and the published SplitMix64 vector."""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere_counts_and_surface(level):
    m = synth.icosphere(level)
    assert m.n == 20 * 4 ** level
    v = m.tri.reshape(-1, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)
    # flat inscribed panels: total area strictly below 4 pi, and centroids inside the sphere
    assert m.area.sum() < 4 * math.pi
    assert np.all(np.linalg.norm(m.centroid, axis=1) < 1.0)
    # outward orientation: normal . centroid > 0
    a, b, c = m.tri[:, 0], m.tri[:, 1], m.tri[:, 2]
    assert np.all(np.einsum("ij,ij->i", np.cross(b - a, c - a), m.centroid) > 0)


def test_icosphere_area_converges_to_4pi():
    errs = [4 * math.pi - synth.icosphere(L).area.sum() for L in range(0, 5)]
    assert all(e > 0 for e in errs)
    ratios = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    assert all(q > 3.0 for q in ratios) and ratios[-1] > 3.9  # O(h^2): -> 4x per level


def test_icosphere_euler_characteristic():
    m = synth.icosphere(2)
    v = np.round(m.tri.reshape(-1, 3), 12)
    verts = {tuple(p) for p in v}
    edges = set()
    for t in np.round(m.tri, 12):
        p = [tuple(x) for x in t]
        for i in range(3):
            edges.add(frozenset((p[i], p[(i + 1) % 3])))
    assert len(verts) - len(edges) + m.n == 2


def test_two_spheres_layout():
    m = synth.two_spheres(1)
    assert m.n == 160
    assert np.all(m.centroid[:80, 0] < 1.0) and np.all(m.centroid[80:, 0] > 2.0)
    b = synth.rhs_two_spheres(m)
    assert b[:80].min() == 1.0 and b[80:].max() == -1.0


def test_cube_and_cube_sphere():
    m = synth.unit_cube(3)
    assert m.n == 108
    assert abs(m.area.sum() - 6.0) < 1e-13
    cs = synth.cube_sphere(4)
    assert cs.n == 192
    assert np.allclose(np.linalg.norm(cs.tri.reshape(-1, 3), axis=1), 1.0)


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (Vigna's reference generator)
    u = synth.splitmix64_uniform(1, 0)[0]
    assert u == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53


def test_normal_columns_moments():
    z = synth.rhs_normal_columns(4096, 4, seed=20191101)
    assert z.shape == (4096, 4) and z.flags["F_CONTIGUOUS"]
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1.0) < 0.05


def test_uneven_batch_specs_range():
    specs = synth.uneven_batch_specs(48)
    assert len(specs) == 48
    ns = [12 * n * n for _, n in specs]
    assert min(ns) >= 1000 and max(ns) <= 21000
    assert {k for k, _ in specs} == {"cube", "sphere"}
