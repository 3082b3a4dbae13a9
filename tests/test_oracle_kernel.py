"""Pins of the oracle's collocation kernel against quadrature of the single-layer
potential (1/4pi) * integral over panel j of 1/|c_i - y| dy (unit permittivity)."""
import math

import numpy as np
from scipy import integrate

import synth


def _self_potential_exact(tri):
    """(1/4pi) * integral over the flat triangle of 1/|c - y| with c its centroid, in
    polar coordinates about c: (1/4pi) * integral_0^{2pi} R(theta) d theta, R the
    distance from c to the boundary along direction theta."""
    a, b, c = tri
    ctr = (a + b + c) / 3.0
    e1 = (b - a) / np.linalg.norm(b - a)
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    e2 = np.cross(nrm, e1)
    P = [np.array([np.dot(p - ctr, e1), np.dot(p - ctr, e2)]) for p in (a, b, c)]

    def R(theta):
        d = np.array([math.cos(theta), math.sin(theta)])
        best = math.inf
        for k in range(3):
            p, q = P[k], P[(k + 1) % 3]
            M = np.array([d, p - q]).T
            try:
                t, s = np.linalg.solve(M, p)
            except np.linalg.LinAlgError:
                continue
            if t > 0 and -1e-12 <= s <= 1 + 1e-12:
                best = min(best, t)
        return best

    angs = sorted(math.atan2(p[1], p[0]) % (2 * math.pi) for p in P)
    pts = angs + [angs[0] + 2 * math.pi]
    total = 0.0
    for k in range(3):
        v, _ = integrate.quad(R, pts[k], pts[k + 1], epsabs=1e-13, epsrel=1e-12, limit=200)
        total += v
    return total / (4 * math.pi)


def _far_potential_quad(x, tri, levels=5):
    """(1/4pi) * integral over the triangle of 1/|x - y| by the centroid rule on
    4**levels congruent sub-triangles."""
    tris = [tri]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nxt
    s = 0.0
    for a, b, c in tris:
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        s += area / np.linalg.norm(x - (a + b + c) / 3)
    return s / (4 * math.pi)


def test_self_term_is_disk_approximation_of_exact_panel_integral(oracle_mod):
    m = synth.icosphere(2)
    for i in (0, 7, 101, 319):
        a_ii = oracle_mod.kernel_entry(m.centroid, m.area, i, i)
        exact = _self_potential_exact(m.tri[i])
        # an equal-area disk over-estimates a near-equilateral triangle by ~2%
        assert 1.0 < a_ii / exact < 1.03, (i, a_ii, exact)


def test_disk_self_term_closed_form(oracle_mod):
    # a single panel whose "area" is that of a unit disk: potential at the centre of a
    # uniformly charged unit disk is (1/4pi) * 2 pi * R = R/2 = 0.5
    c = np.zeros((1, 3))
    area = np.array([math.pi])
    assert abs(oracle_mod.kernel_entry(c, area, 0, 0) - 0.5) < 1e-15


def test_far_entries_match_panel_quadrature(oracle_mod):
    m = synth.icosphere(3)
    rng = np.random.default_rng(1)
    h = math.sqrt(m.area.mean())
    checked = 0
    for _ in range(200):
        i, j = rng.integers(0, m.n, 2)
        r = np.linalg.norm(m.centroid[i] - m.centroid[j])
        if r < 10 * h:
            continue
        a_ij = oracle_mod.kernel_entry(m.centroid, m.area, i, j)
        q = _far_potential_quad(m.centroid[i], m.tri[j], levels=3)
        assert abs(a_ij / q - 1.0) < 2e-3, (i, j, a_ij, q)
        checked += 1
    assert checked > 50


def test_dense_matrix_uses_source_panel_area(oracle_mod):
    # the one-point rule integrates over panel j: a_ij * 4 pi r = area_j exactly
    m = synth.icosphere(1)
    A = oracle_mod.dense_matrix(m.centroid, m.area)
    i, j = 3, 50
    r = np.linalg.norm(m.centroid[i] - m.centroid[j])
    q = _far_potential_quad(m.centroid[i], m.tri[j], levels=6)
    assert abs(A[i, j] - q) / q < 0.05          # near pair: one-point rule within a few %
    assert abs(A[i, j] * 4 * math.pi * r / m.area[j] - 1.0) < 1e-14
